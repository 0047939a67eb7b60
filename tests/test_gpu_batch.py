"""Ensembles (hydro_batch_*): independent problems on uneven grids advanced together in one graph launch.

Each member must evolve exactly as the same problem run alone through the single-problem path (same
per-cell arithmetic, whatever tile shape the autotuner picks), and match the FP64 oracle after a step.
"""
import numpy as np
import pytest

import hydro_problems as hp
import oracle

pytestmark = pytest.mark.gpu
NG = 4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6883_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _members(seed=0):
    g = np.random.default_rng(seed)
    shapes = [(16, 16), (37, 21), (64, 64), (48, 80), (5, 3), (64, 64), (100, 30)]
    return [hp.quad(nx, ny, rng=g) for nx, ny in shapes]


def _alone(pr, precision, nsteps):
    from paper_1306_6883_gb300.solver import Solver, params_for
    s = Solver(params_for(pr, precision), pr.U)
    s.advance(nsteps)
    out = s.state_numpy()
    t, n = s.time()
    s.close()
    return out, t


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("tune", [False, True])
def test_members_evolve_exactly_as_alone(precision, tune):
    from paper_1306_6883_gb300.solver import Ensemble, params_for
    probs = _members()
    e = Ensemble([params_for(p, precision) for p in probs], [p.U for p in probs])
    if tune:
        shapes = e.autotune(reps=2)
        assert len(shapes) == len(e.classes())
    e.run(6)
    st, stats = e.status()
    assert st == 0 and stats[0] > 0
    for i, pr in enumerate(probs):
        ref, t_ref = _alone(pr, precision, 6)
        got = e.state_numpy(i)[:, NG:-NG, NG:-NG]
        ref = ref[:, NG:-NG, NG:-NG]
        t, n = e.time(i)
        assert n == 6
        if precision == 0:  # FP64 kernels round every operation on its own: bit for bit
            np.testing.assert_array_equal(got, ref)
            assert t == t_ref
        else:  # FP32 kernels compiled apart may fuse different multiply-adds: equal to FP32 rounding
            scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
            assert np.all(np.abs(got - ref) <= 2.0 ** -24 * 256 * scale), np.abs(got - ref).max()
            assert t == pytest.approx(t_ref, rel=2.0 ** -24 * 16)
    e.close()


def test_graph_launch_equals_direct_launches():
    from paper_1306_6883_gb300.solver import Ensemble, params_for
    probs = _members(seed=3)
    a = Ensemble([params_for(p, 1) for p in probs], [p.U for p in probs])
    b = Ensemble([params_for(p, 1) for p in probs], [p.U for p in probs])
    a.run(5, use_graph=True)
    a.run(5, use_graph=True)   # the cached graph of the other parity
    b.run(10, use_graph=False)
    for i in range(len(probs)):
        np.testing.assert_array_equal(a.state_numpy(i), b.state_numpy(i))
    a.close()
    b.close()


def test_member_matches_the_oracle_after_one_step():
    from paper_1306_6883_gb300.solver import Ensemble, params_for
    probs = _members(seed=5)
    e = Ensemble([params_for(p, 0) for p in probs], [p.U for p in probs])
    e.run(1)
    for i, pr in enumerate(probs):
        po = oracle.params(pr.nx, pr.ny, bc=pr.bc)
        U = pr.U.copy()
        oracle.fill_ghost(po, U)
        oracle.step(po, U, oracle.cfl_dt(po, U))
        got = e.state_numpy(i)[:, NG:-NG, NG:-NG]
        ref = U[:, NG:-NG, NG:-NG]
        scale = np.abs(ref).reshape(4, -1).max(axis=1)[:, None, None]
        assert np.all(np.abs(got - ref) <= 1e-12 * scale)
    e.close()


def test_member_totals_are_conserved_with_periodic_boundaries():
    from paper_1306_6883_gb300.solver import Ensemble, params_for
    probs = [hp.kh(32, 32, seed=1), hp.kh(64, 48, seed=2), hp.kh(16, 80, seed=3)]
    e = Ensemble([params_for(p, 0) for p in probs], [p.U for p in probs])
    t0 = [np.array(e.totals(i)) for i in range(3)]
    e.run(20)
    for i, pr in enumerate(probs):
        t1 = np.array(e.totals(i))
        scale = np.abs(pr.U[:, NG:-NG, NG:-NG]).sum(axis=(1, 2)) / (pr.nx * pr.ny)
        assert np.all(np.abs(t1 - t0[i]) <= 1e-13 * scale)
    e.close()


def test_ensemble_sizes_of_the_256_member_workload():
    sizes = hp.ensemble_sizes(256, seed=0)
    assert len(sizes) == 256 and set(sizes) <= {64, 128, 256, 512}
    assert len(set(sizes)) == 4
