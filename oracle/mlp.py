"""FP64 reference of the learned star-pressure proposal -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this module.  Plain numpy, FP64.

The proposal (not in the paper; it feeds the two-shock iteration of §3.2 a starting pressure) is an MLP
6 -> 64 -> 64 -> 1 with ReLU on the hidden layers.  Its six inputs are the left and right (rho, u_n, p) of
a face in reference units that use the scaling symmetry of the Euler equations:
    rho_ref = sqrt(rho_L rho_R), p_ref = sqrt(p_L p_R), c_ref = sqrt(p_ref / rho_ref), u_mean = (u_L + u_R)/2,
    x = (ln(rho_L/rho_ref), (u_L - u_mean)/c_ref, ln(p_L/p_ref), ln(rho_R/rho_ref), (u_R - u_mean)/c_ref,
         ln(p_R/p_ref)),
and its output is y = ln(p*/p_ref), so the proposal is p0 = p_ref exp(y).  The training loss is the mean
squared error of y over a minibatch.

Parameter vector layout (4673 float values), shared by the CUDA kernels:
    W1 [64][6], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]
(W[i][k] multiplies input k into output i).
"""
import numpy as np

NIN, NH = 6, 64
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def features(rl, ul, pl, rr, ur, pr):
    """Reference-unit inputs and the reference pressure of faces (arrays of equal shape)."""
    rl, ul, pl, rr, ur, pr = (np.asarray(a, dtype=np.float64) for a in (rl, ul, pl, rr, ur, pr))
    rho_ref = np.sqrt(rl * rr)
    p_ref = np.sqrt(pl * pr)
    c_ref = np.sqrt(p_ref / rho_ref)
    um = 0.5 * (ul + ur)
    x = np.stack([np.log(rl / rho_ref), (ul - um) / c_ref, np.log(pl / p_ref),
                  np.log(rr / rho_ref), (ur - um) / c_ref, np.log(pr / p_ref)], axis=-1)
    return x, p_ref


def forward(theta, x):
    """Network output y for inputs x [n, 6]; returns (y, cache)."""
    P = unpack(theta)
    z1 = x @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"] + P["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss(theta, x, t):
    y, _ = forward(theta, x)
    return float(np.mean((y - t) ** 2))


def gradient(theta, x, t):
    """Analytic gradient of the mean squared error (backpropagation through the three layers)."""
    P = unpack(theta)
    y, (x, z1, h1, z2, h2) = forward(theta, x)
    n = x.shape[0]
    dy = 2.0 * (y - t) / n
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, P["W3"]) * (z2 > 0.0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * (z1 > 0.0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def init(seed=0):
    """He-normal weights, zero biases (the CUDA initialiser draws its own numbers; tests pass theta in)."""
    g = np.random.default_rng(seed)
    return pack({"W1": g.normal(0, np.sqrt(2.0 / NIN), (NH, NIN)), "b1": np.zeros(NH),
                 "W2": g.normal(0, np.sqrt(2.0 / NH), (NH, NH)), "b2": np.zeros(NH),
                 "W3": g.normal(0, np.sqrt(1.0 / NH), NH), "b3": np.zeros(1)})
