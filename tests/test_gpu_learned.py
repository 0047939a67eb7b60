"""The learned starting pressure of the two-shock iteration: harvest, GPU training kernels (gradients checked
against the FP64 reference MLP), tensor-core inference, and the CTU step that uses it -- whose answer must
stay the method's (the iteration still converges to the same tolerance)."""
import numpy as np
import pytest

import hydro_problems as hp
import oracle
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
NG = 4


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6883_gb300 import build
    build.build()
    t.cuda.set_device(0)
    return t


def _random_faces(n, seed):
    """Synthetic Riemann problems with their converged star pressures from the FP64 oracle."""
    rng = np.random.default_rng(seed)
    P = oracle.params(8, 8, riemann_tol=1e-12)
    out = np.zeros((n, 8), dtype=np.float32)
    k = 0
    while k < n:
        rl, rr = np.exp(rng.uniform(np.log(0.1), np.log(2.0), 2))
        pl, pr = np.exp(rng.uniform(np.log(0.01), np.log(10.0), 2))
        ul, ur = rng.uniform(-1.5, 1.5, 2)
        L = np.float32([rl, ul, 0.0, pl]).astype(np.float64)
        R = np.float32([rr, ur, 0.0, pr]).astype(np.float64)
        r = oracle.riemann(P, L, R)
        if not r["converged"] or r["pstar"] < 1e-6:
            continue
        out[k] = [L[0], L[1], L[3], R[0], R[1], R[3], r["pstar"], r["iters"]]
        k += 1
    return out


def _oracle_xt(s):
    x, pref = omlp.features(*[s[:, i].astype(np.float64) for i in range(6)])
    return x, np.log(s[:, 6].astype(np.float64) / pref)


def test_gpu_gradient_matches_the_fp64_reference(torch):
    from paper_1306_6883_gb300.solver import Model
    s = _random_faces(300, seed=1)
    m = Model(seed=7)
    theta = m.weights().astype(np.float64)
    d = torch.from_numpy(s).cuda()
    g_gpu, loss_gpu = m.gradient(d)
    x, t = _oracle_xt(s)
    g_ref = omlp.gradient(theta, x, t)
    assert loss_gpu == pytest.approx(omlp.loss(theta, x, t), rel=1e-4)
    scale = np.abs(g_ref).max()
    assert np.abs(g_gpu - g_ref).max() <= 1e-3 * scale, np.abs(g_gpu - g_ref).max() / scale
    # every parameter block is exercised
    for lo, hi in ((0, 384), (384, 448), (448, 4544), (4544, 4608), (4608, 4672), (4672, 4673)):
        assert np.abs(g_gpu[lo:hi]).max() > 0
    m.close()


def test_predictions_match_the_reference_forward(torch):
    from paper_1306_6883_gb300.solver import Model
    s = _random_faces(500, seed=2)
    m = Model(seed=3)
    theta = m.weights().astype(np.float64)
    d = torch.from_numpy(s).cuda()
    x, _ = _oracle_xt(s)
    y_ref, _ = omlp.forward(theta, x)
    y32 = m.predict(d).cpu().numpy()
    assert np.abs(y32 - y_ref).max() <= 1e-4 * (1 + np.abs(y_ref).max())
    # BF16 weights and activations: about 3 significant digits
    ytc = m.predict(d, tensor_cores=True).cpu().numpy()
    assert np.abs(ytc - y_ref).max() <= 0.03 * (1 + np.abs(y_ref).max())
    m.close()


def test_training_lowers_the_loss_and_proposes_good_starts(torch):
    from paper_1306_6883_gb300.solver import Model
    train = torch.from_numpy(_random_faces(20000, seed=3)).cuda()
    held = _random_faces(2000, seed=4)
    m = Model(seed=5)
    _, loss0 = m.gradient(torch.from_numpy(held).cuda())
    m.train(train, steps=1500, batch=1024, lr=2e-3, seed=9)
    _, loss1 = m.gradient(torch.from_numpy(held).cuda())
    assert loss1 < 0.05 * loss0, (loss0, loss1)
    # the trained proposal is closer to p* than the acoustic estimate on held-out faces
    x, t = _oracle_xt(held)
    y = m.predict(torch.from_numpy(held).cuda(), tensor_cores=True).cpu().numpy()
    P = oracle.params(8, 8)
    ac = []
    for r in held:
        cl = np.sqrt(1.4 * r[2] * r[0])
        cr = np.sqrt(1.4 * r[5] * r[3])
        p0 = max((cr * r[2] + cl * r[5] + cl * cr * (r[1] - r[4])) / (cl + cr), 1e-20)
        ac.append(p0)
    _, pref = omlp.features(*[held[:, i].astype(np.float64) for i in range(6)])
    err_ml = np.abs(y - t)
    err_ac = np.abs(np.log(np.array(ac) / pref) - t)
    assert np.median(err_ml) < np.median(err_ac), (np.median(err_ml), np.median(err_ac))
    m.close()


def test_harvest_records_valid_riemann_problems(torch):
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Harvest, Solver, params_for
    pr = hp.sod(64, 64)
    s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
    hv = Harvest(s, capacity=20000, rate=0.25)
    s.advance(5)
    st, stats = s.status()
    smp = hv.samples().cpu().numpy()
    n_total = int(hv.count.item())
    # about a quarter of the 5 steps' solves were sampled
    assert 0.2 * stats[0] < n_total < 0.3 * stats[0]
    assert smp.shape[0] == min(n_total, 20000) and np.all(np.isfinite(smp))
    P = oracle.params(8, 8, riemann_tol=1e-12)
    for r in smp[:: max(1, len(smp) // 200)]:
        res = oracle.riemann(P, [r[0], r[1], 0.0, r[2]], [r[3], r[4], 0.0, r[5]])
        assert r[6] == pytest.approx(res["pstar"], rel=2e-5, abs=1e-12)
    s.close()


def test_harvest_gate_keeps_every_strong_face(torch):
    # with a negligible random rate, the gated harvest records exactly the faces past the gate: every
    # record is a strong face, and a run with the gate records more of them than the random rate alone
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Harvest, Solver, params_for
    counts = {}
    for gated in (False, True):
        pr = hp.sod(64, 64)
        s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
        hv = Harvest(s, capacity=200000, rate=1e-9)
        if gated:
            H.hydro_set_harvest_gate(s.ctx, 0.35, 1.0)
        s.advance(5)
        s.status()
        smp = hv.samples().cpu().numpy().astype(np.float32)
        counts[gated] = smp.shape[0]
        if gated:
            pl, pr_, du = smp[:, 2], smp[:, 5], smp[:, 1] - smp[:, 4]
            ratio, u4 = np.float32(np.exp(0.7)), np.float32(1.0)
            strong = (np.maximum(pl, pr_) >= ratio * np.minimum(pl, pr_)) | \
                     ((du * du) * (du * du) * (smp[:, 0] * smp[:, 3]) >= u4 * (pl * pr_))
            assert smp.shape[0] > 0 and np.all(strong)
        s.close()
    assert counts[True] > counts[False]
    with pytest.raises(H.HydroError):
        pr = hp.sod(16, 16)
        s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
        try:
            H.hydro_set_harvest_gate(s.ctx, 0.35, 0.0)  # half-set gate
        finally:
            s.close()


def _step(pr, learned_model=None, nsteps=1):
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for
    s = Solver(params_for(pr, H.HYDRO_FP32, use_learned_guess=1 if learned_model else 0), pr.U)
    if learned_model:
        H.hydro_set_riemann_model(s.ctx, learned_model.m)
    s.fill_ghost()
    Uin = s.state_numpy()
    dt = s.cfl_dt()
    s.step(dt)
    if nsteps > 1:
        s.advance(nsteps - 1)
    st, stats = s.status(raise_on_error=False)
    out = s.state_numpy()
    s.close()
    return Uin, out, dt, st, stats


def test_learned_start_leaves_the_answer_to_the_method(torch):
    from paper_1306_6883_gb300.solver import Model
    m = Model(seed=11)
    m.train(torch.from_numpy(_random_faces(20000, seed=6)).cuda(), steps=800, batch=1024, lr=2e-3, seed=3)
    m.set_gate(0.0, 0.0)  # every warp evaluates the network
    for pr in (hp.quad(96, 80, seed=12), hp.sedov(96, 96, r_init=0.05), hp.sod(64, 64)):
        Uin, plain, dt, st0, s0 = _step(pr)
        _, learned, dt1, st1, s1 = _step(pr, m)
        assert st0 == 0 and st1 == 0 and dt == dt1
        # same converged fluxes to the FP32 tolerance: agreement with each other and with the oracle
        ref = Uin.astype(np.float64)
        po = oracle.params(pr.nx, pr.ny, bc=pr.bc)
        oracle.fill_ghost(po, ref)
        oracle.step(po, ref, dt)
        for got in (plain, learned):
            g = got[:, NG:-NG, NG:-NG].astype(np.float64)
            r = ref[:, NG:-NG, NG:-NG]
            scale = np.where(np.abs(r).reshape(4, -1).max(axis=1) > 0, np.abs(r).reshape(4, -1).max(axis=1), 1.0)
            assert np.all(np.abs(g - r).reshape(4, -1).max(axis=1) <= 2e-5 * scale)
        assert s1[0] == s0[0] and s1[2] == 0
    m.close()


def test_an_untrained_network_does_not_change_the_answer(torch):
    # whatever the start, the iteration converges to the same star pressure (same result, no failures)
    from paper_1306_6883_gb300.solver import Model
    m = Model(seed=13)
    m.set_gate(0.0, 0.0)
    pr = hp.quad(64, 64, seed=14)
    _, plain, _, _, s0 = _step(pr)
    _, learned, _, st, s1 = _step(pr, m)
    assert st == 0 and s1[2] == 0 and s1[0] == s0[0]
    scale = np.abs(plain[:, NG:-NG, NG:-NG]).reshape(4, -1).max(axis=1)
    err = np.abs(learned - plain)[:, NG:-NG, NG:-NG].reshape(4, -1).max(axis=1) / np.where(scale > 0, scale, 1)
    assert np.all(err <= 4e-5), err
    m.close()


def test_learned_mode_requires_a_model(torch):
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for
    pr = hp.sod(16, 8)
    s = Solver(params_for(pr, H.HYDRO_FP32, use_learned_guess=1), pr.U)
    s.fill_ghost()
    with pytest.raises(H.HydroError) as e:
        s.step(s.cfl_dt())
    assert e.value.status == H.HYDRO_EINVAL
    s.close()


def test_fused_learned_step_equals_the_separate_passes(torch):
    # hydro_step_fused on a learned context is one launch (boundary map, CTU step started from the network,
    # CFL dt of the new state); it must give the state of ghost fill + dt + hydro_step to float rounding (two
    # compilations of the same tile code) and stay within the FP32 bound of the oracle's step
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Model, Solver, params_for
    m = Model(seed=21)
    m.train(torch.from_numpy(_random_faces(20000, seed=22)).cuda(), steps=600, batch=1024, lr=2e-3, seed=4)
    m.set_gate(0.0, 0.0)  # every warp evaluates the network
    for pr in (hp.quad(96, 80, seed=23), hp.sod(64, 48)):
        a = Solver(params_for(pr, H.HYDRO_FP32, use_learned_guess=1), pr.U)
        b = Solver(params_for(pr, H.HYDRO_FP32, use_learned_guess=1), pr.U)
        H.hydro_set_riemann_model(a.ctx, m.m)
        H.hydro_set_riemann_model(b.ctx, m.m)
        for _ in range(4):
            a.fill_ghost()
            a.step(a.cfl_dt())
            b.step_fused()
        sa, _ = a.status()
        sb, stats = b.status()
        assert sa == 0 and sb == 0 and stats[2] == 0
        A = a.interior().astype(np.float64)
        B = b.interior().astype(np.float64)
        # each field's magnitude, floored at 1e-3 of the largest (the Sod tube's rho v is round-off only)
        scale = np.maximum(np.abs(A).reshape(4, -1).max(axis=1), 1e-3 * np.abs(A).max())
        assert np.all(np.abs(A - B).reshape(4, -1).max(axis=1) <= 1e-4 * scale)
        a.close()
        b.close()
        # one fused learned step against the oracle's step from the same state
        c = Solver(params_for(pr, H.HYDRO_FP32, use_learned_guess=1), pr.U)
        H.hydro_set_riemann_model(c.ctx, m.m)
        Uin = c.state_numpy().astype(np.float64)
        c.step_fused()
        t, _ = c.time()
        got = c.interior().astype(np.float64)
        c.close()
        po = oracle.params(pr.nx, pr.ny, bc=pr.bc)
        oracle.fill_ghost(po, Uin)
        oracle.step(po, Uin, t)
        ref = Uin[:, NG:-NG, NG:-NG]
        scale = np.maximum(np.abs(ref).reshape(4, -1).max(axis=1), 1e-3 * np.abs(ref).max())
        assert np.all(np.abs(got - ref).reshape(4, -1).max(axis=1) <= 2e-5 * scale)
    m.close()


def _quads(seed):
    g = np.random.default_rng(seed)
    return [hp.quad(nx, ny, rng=g) for nx, ny in ((64, 64), (37, 21), (128, 96), (16, 16), (64, 64))]


def test_learned_ensemble_members_evolve_as_alone(torch):
    # every member of an ensemble started from the network evolves as the same problem run alone with the
    # same network (the batched persistent kernel and the single-problem fused kernel are two compilations of
    # the same tile code: equal to float rounding), and stays within the FP32 bound of the oracle after a step
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Ensemble, Model, Solver, params_for
    m = Model(seed=31)
    m.train(torch.from_numpy(_random_faces(20000, seed=32)).cuda(), steps=600, batch=1024, lr=2e-3, seed=5)
    m.set_gate(0.0, 0.0)
    probs = _quads(33)
    for tune in (False, True):
        e = Ensemble([params_for(p, H.HYDRO_FP32, use_learned_guess=1) for p in probs], [p.U for p in probs])
        e.set_model(m)
        if tune:
            e.autotune(reps=1)
        e.run(5)
        st, stats = e.status()
        assert st == 0 and stats[0] > 0 and stats[2] == 0
        for i, pr in enumerate(probs):
            s = Solver(params_for(pr, H.HYDRO_FP32, use_learned_guess=1), pr.U)
            H.hydro_set_riemann_model(s.ctx, m.m)
            s.advance(5)
            ref = s.interior().astype(np.float64)
            t_ref, _ = s.time()
            s.close()
            got = e.state_numpy(i)[:, NG:-NG, NG:-NG].astype(np.float64)
            scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
            assert np.all(np.abs(got - ref) <= 2.0 ** -24 * 256 * scale), np.abs(got - ref).max()
            t, n = e.time(i)
            assert n == 5 and t == pytest.approx(t_ref, rel=2.0 ** -24 * 16)
        e.close()
    # one step of each member against the oracle
    e = Ensemble([params_for(p, H.HYDRO_FP32, use_learned_guess=1) for p in probs], [p.U for p in probs])
    e.set_model(m)
    e.run(1)
    for i, pr in enumerate(probs):
        t, _ = e.time(i)
        U = pr.U.astype(np.float32).astype(np.float64)
        po = oracle.params(pr.nx, pr.ny, bc=pr.bc)
        oracle.fill_ghost(po, U)
        oracle.step(po, U, t)
        got = e.state_numpy(i)[:, NG:-NG, NG:-NG].astype(np.float64)
        ref = U[:, NG:-NG, NG:-NG]
        scale = np.abs(ref).reshape(4, -1).max(axis=1)
        assert np.all(np.abs(got - ref).reshape(4, -1).max(axis=1) <= 2e-5 * scale)
    e.close()
    m.close()


def test_learned_ensemble_needs_its_model(torch):
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Ensemble, Model, params_for
    probs = _quads(41)[:2]
    m = Model(seed=1)
    # members created without the learned start refuse a model
    plain = Ensemble([params_for(p, H.HYDRO_FP32) for p in probs], [p.U for p in probs])
    with pytest.raises(H.HydroError) as ex:
        plain.set_model(m)
    assert ex.value.status == H.HYDRO_EINVAL
    plain.close()
    # learned members refuse to run without one, and mixed members are rejected at creation
    e = Ensemble([params_for(p, H.HYDRO_FP32, use_learned_guess=1) for p in probs], [p.U for p in probs])
    with pytest.raises(H.HydroError):
        e.run(1)
    e.set_model(m)
    e.run(1)
    e.set_model(None)
    with pytest.raises(H.HydroError):
        e.run(1)
    e.close()
    with pytest.raises(H.HydroError):
        Ensemble([params_for(probs[0], H.HYDRO_FP32, use_learned_guess=1), params_for(probs[1], H.HYDRO_FP32)],
                 [p.U for p in probs])
    m.close()


def test_sedov_8192_learned_fp32_error_against_fp64(torch):
    # the largest workload: the Sedov blast on 8192^2 cells with 1 % density noise, FP32 with the learned
    # start (default gate) against the FP64 run, which is the oracle's bit for bit, after 25 fused steps from
    # the same state.  Observed on GB300 (25 steps): L1 relative 2.2e-8 (rho), 4.0e-7 (rho u, rho v), 5.8e-8
    # (E); max relative 9.1e-7, 8.3e-7, 8.4e-7, 7.0e-7.  Bounds 6-8x those.
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Model, Solver, params_for
    m = Model(seed=21)
    m.train(torch.from_numpy(_random_faces(20000, seed=22)).cuda(), steps=800, batch=1024, lr=2e-3, seed=23)
    pr = hp.sedov(8192, 8192, density_noise=0.01)
    out = {}
    for prec in (H.HYDRO_FP64, H.HYDRO_FP32):
        learned = prec == H.HYDRO_FP32
        s = Solver(params_for(pr, prec, use_learned_guess=1 if learned else 0), pr.U)
        if learned:
            H.hydro_set_riemann_model(s.ctx, m.m)
        s.advance(25)
        st, stats = s.status()
        assert st == 0 and stats[2] == 0
        out[prec] = s.interior()
        s.close()
    m.close()
    l1, mx = np.zeros(4), np.zeros(4)
    for k in range(4):  # field by field: the 8192^2 arrays are 0.5 GB each in double
        b = out[H.HYDRO_FP64][k]
        d = np.abs(out[H.HYDRO_FP32][k].astype(np.float64) - b)
        l1[k] = d.sum() / np.abs(b).sum()
        mx[k] = d.max() / np.abs(b).max()
    assert np.all(l1 <= np.array([1.6e-7, 2.8e-6, 2.8e-6, 4e-7])), l1
    assert np.all(mx <= np.array([6e-6, 6e-6, 6e-6, 5e-6])), mx
