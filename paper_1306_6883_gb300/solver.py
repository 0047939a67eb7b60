"""Convenience wrapper around the C ABI with PyTorch-owned device buffers (memory and stream only).

    s = Solver(params, U0_numpy)      # U0: (4, ny+2ng, nx+2ng) float64 array, dense layout
    s.fill_ghost(); dt = s.cfl_dt(); s.step(dt)
    U = s.state_numpy()

Every operation is one C-ABI call; no arithmetic of the method happens here.
"""
import numpy as np
import torch

from . import hydro as H


class Solver:
    def __init__(self, params, U0=None, stream=None, device="cuda"):
        self.p = params
        self.dtype = torch.float32 if params.precision == H.HYDRO_FP32 else torch.float64
        self.np_dtype = np.float32 if params.precision == H.HYDRO_FP32 else np.float64
        self.pitch = H.state_pitch(params)
        if self.pitch == 0:
            raise H.HydroError(H.HYDRO_EINVAL, "invalid parameters")
        self.NX = params.nx + 2 * params.ng
        self.NY = params.ny + 2 * params.ng
        n = 4 * self.NY * self.pitch
        self.bufs = [torch.zeros(n, dtype=self.dtype, device=device) for _ in range(2)]
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.ctx = H.hydro_init(params, self.bufs[0].data_ptr(), self.bufs[1].data_ptr(), self.stream.cuda_stream)
        if U0 is not None:
            self.set_state(U0)

    def close(self):
        if self.ctx is not None:
            H.hydro_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the C-ABI calls
    def fill_ghost(self):
        H.hydro_fill_ghost(self.ctx)

    def cfl_dt(self):
        return H.hydro_cfl_dt(self.ctx)

    def step(self, dt):
        H.hydro_step(self.ctx, dt)

    def advance(self, nsteps, tmax=0.0):
        H.hydro_advance(self.ctx, nsteps, tmax)

    def cfl_dt_async(self, tmax=0.0):
        H.hydro_cfl_dt_async(self.ctx, tmax)

    def step_device_dt(self):
        H.hydro_step_device_dt(self.ctx)

    def step_fused(self, tmax=0.0):
        H.hydro_step_fused(self.ctx, tmax)

    def upload(self, host_tensor):
        """Enqueue a copy of a pinned host tensor (4, NY, NX) into the current state."""
        H.hydro_upload(self.ctx, host_tensor.data_ptr())

    def download(self, host_tensor):
        H.hydro_download(self.ctx, host_tensor.data_ptr())

    def step_host(self, host_in, host_out, tmax=0.0, chained=False):
        """One step from a pinned host tensor to another (upload, fused step, download, overlapped).  With
        chained=True, host_in continuing the previous call's host_out unchanged, the step reuses the time
        step that call reduced, and the upload overlaps the step."""
        fn = H.hydro_step_host_chained if chained else H.hydro_step_host
        fn(self.ctx, host_in.data_ptr(), host_out.data_ptr(), tmax)

    def time(self):
        return H.hydro_get_time(self.ctx)

    def totals(self):
        return H.hydro_conserved_totals(self.ctx)

    def status(self, raise_on_error=True):
        return H.hydro_sync_status(self.ctx, raise_on_error)

    # ---- state access
    def current(self):
        """Torch view (4, NY, pitch) of the buffer that holds the current state."""
        ptr = H.hydro_state(self.ctx)
        buf = self.bufs[0] if ptr == self.bufs[0].data_ptr() else self.bufs[1]
        return buf.view(4, self.NY, self.pitch)

    def set_state(self, U):
        U = np.ascontiguousarray(U, dtype=self.np_dtype)
        assert U.shape == (4, self.NY, self.NX), U.shape
        host = torch.from_numpy(U).pin_memory()
        H.hydro_upload(self.ctx, host.data_ptr())
        self.stream.synchronize()

    def state_numpy(self):
        out = torch.empty((4, self.NY, self.NX), dtype=self.dtype).pin_memory()
        H.hydro_download(self.ctx, out.data_ptr())
        return out.numpy().copy()

    def interior(self):
        g = self.p.ng
        return self.state_numpy()[:, g:-g, g:-g]


def params_for(problem, precision=H.HYDRO_FP64, **kw):
    """C-ABI parameters for a hydro_problems.Problem."""
    xmin, xmax, ymin, ymax = problem.domain
    return H.default_params(problem.nx, problem.ny, precision, bc=problem.bc, gamma=problem.gamma, cfl=problem.cfl,
                            xmin=xmin, xmax=xmax, ymin=ymin, ymax=ymax, ng=problem.ng,
                            grav=getattr(problem, "grav", 0.0), **kw)


class Ensemble:
    """Independent problems advanced together through the hydro_batch_* calls (PyTorch owns the buffers).

        e = Ensemble([params_for(p, H.HYDRO_FP32) for p in problems], [p.U for p in problems])
        e.autotune(); e.run(100)
    """

    def __init__(self, params_list, states, stream=None, device="cuda"):
        self.params = list(params_list)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.bufs, self.shapes = [], []
        for p in self.params:
            dt = torch.float32 if p.precision == H.HYDRO_FP32 else torch.float64
            pitch = H.state_pitch(p)
            NX, NY = p.nx + 2 * p.ng, p.ny + 2 * p.ng
            self.shapes.append((NY, NX, pitch, dt))
            self.bufs.append([torch.zeros(4 * NY * pitch, dtype=dt, device=device) for _ in range(2)])
        for i, U in enumerate(states):
            NY, NX, pitch, dt = self.shapes[i]
            view = self.bufs[i][0].view(4, NY, pitch)
            view[:, :, :NX].copy_(torch.from_numpy(np.ascontiguousarray(U)).to(dt))
        torch.cuda.synchronize()
        self.b = H.hydro_batch_create(self.params, [x[0].data_ptr() for x in self.bufs],
                                      [x[1].data_ptr() for x in self.bufs], self.stream.cuda_stream)

    def close(self):
        if self.b is not None:
            H.hydro_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, reps=3):
        return H.hydro_batch_autotune(self.b, reps)

    def set_model(self, model):
        """Start every member's Riemann iterations from `model` (a Model; the members need
        use_learned_guess = 1), or from the acoustic estimate again with None."""
        H.hydro_batch_set_riemann_model(self.b, model.m if model is not None else None)

    def classes(self):
        return H.hydro_batch_classes(self.b)

    def run(self, nsteps, use_graph=True):
        H.hydro_batch_run(self.b, nsteps, use_graph)

    def time(self, i):
        return H.hydro_batch_get_time(self.b, i)

    def status(self, raise_on_error=True):
        return H.hydro_batch_sync_status(self.b, raise_on_error)

    def totals(self, i):
        return H.hydro_batch_conserved_totals(self.b, i)

    def state_numpy(self, i):
        NY, NX, pitch, dt = self.shapes[i]
        ptr = H.hydro_batch_state(self.b, i)
        buf = self.bufs[i][0] if ptr == self.bufs[i][0].data_ptr() else self.bufs[i][1]
        torch.cuda.synchronize()
        return buf.view(4, NY, pitch)[:, :, :NX].cpu().numpy().copy()


class Model:
    """The learned starting-pressure network (hydro_mlp_*), trained on the GPU by the library's kernels."""

    def __init__(self, seed=0, stream=None, device="cuda"):
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.m = H.hydro_mlp_create(seed, self.stream.cuda_stream)

    def close(self):
        if self.m is not None:
            H.hydro_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weights(self):
        return H.hydro_mlp_get_weights(self.m)

    def set_weights(self, theta):
        H.hydro_mlp_set_weights(self.m, theta)

    def set_gate(self, gate_dp, gate_du):
        H.hydro_mlp_set_gate(self.m, gate_dp, gate_du)

    def gradient(self, samples):
        """samples: CUDA float32 tensor [n, 8]."""
        return H.hydro_mlp_gradient(self.m, samples.data_ptr(), samples.shape[0])

    def train(self, samples, steps, batch=4096, lr=1e-3, seed=1):
        return H.hydro_mlp_train(self.m, samples.data_ptr(), samples.shape[0], steps, batch, lr, seed)

    def predict(self, samples, tensor_cores=False):
        out = torch.empty(samples.shape[0], dtype=torch.float32, device=samples.device)
        H.hydro_mlp_predict(self.m, samples.data_ptr(), samples.shape[0], tensor_cores, out.data_ptr())
        return out


class Harvest:
    """Device buffer that records Riemann problems (inputs, p*, iterations) during a Solver's steps."""

    def __init__(self, solver, capacity, rate):
        self.solver = solver
        self.buf = torch.zeros((capacity, 8), dtype=torch.float32, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int64, device="cuda")
        H.hydro_set_harvest(solver.ctx, self.buf.data_ptr(), capacity, rate, self.count.data_ptr())

    def stop(self):
        H.hydro_set_harvest(self.solver.ctx, 0, 0, 0.0, 0)

    def samples(self):
        n = min(int(self.count.item()), self.buf.shape[0])
        return self.buf[:n]
