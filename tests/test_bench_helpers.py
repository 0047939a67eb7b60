"""Host-side helpers of bench.py that need no GPU: the exact-time driver loop, the traffic figure's source
check, the roofline arithmetic and the FP32-vs-FP64 error summary."""
import os

import numpy as np
import pytest

import bench


class _FakeSolver:
    """A solver whose device loop takes steps of fixed length dt, the last one clamped to land on tmax (as the
    fused step's dt clamp does), and counts every step it is asked for."""

    def __init__(self, dt, stall=False):
        self.t, self.n, self.dt, self.stall = 0.0, 0, dt, stall

    def time(self):
        return self.t, self.n

    def advance(self, k, tmax):
        for _ in range(k):
            step = 0.0 if self.stall else min(self.dt, tmax - self.t)
            self.t += step
            self.n += 1


@pytest.mark.parametrize("dt,tmax", [(0.01, 0.1), (0.003, 0.1), (1e-4, 0.05), (0.2, 0.1)])
def test_advance_to_stops_on_the_step_that_reaches_tmax(dt, tmax):
    s = _FakeSolver(dt)
    n = bench._advance_to(s, tmax)
    expect = int(np.ceil(tmax / dt - 1e-9))
    assert n == expect, (n, expect)
    assert s.t == pytest.approx(tmax, rel=1e-12)


def test_advance_to_refuses_a_stalled_clock():
    with pytest.raises(RuntimeError):
        bench._advance_to(_FakeSolver(0.01, stall=True), 0.1)


def test_traffic_figure_needs_the_captured_sources(tmp_path, monkeypatch):
    prof = tmp_path / "p.md"
    good = bench.kernel_sources_sha256()
    prof.write_text(f"    traffic_bytes_per_launch: 12345\n    sources_sha256: {good}\n")
    monkeypatch.setitem(bench.TRAFFIC_PROFILES, "t", str(prof))  # an absolute path: read as it is
    assert bench.read_traffic("t")[0] == 12345
    prof.write_text(f"    traffic_bytes_per_launch: 12345\n    sources_sha256: {'0' * 64}\n")
    val, note = bench.read_traffic("t")
    assert val is None and "changed" in note
    prof.write_text("no figure here\n")
    assert bench.read_traffic("t")[0] is None


def test_roofline_arithmetic():
    r = bench.roofline("fp32", 1_000_000, 1.0, 1.0, "k")
    flops = bench.FLOPS_BASE + bench.FLOPS_PER_ITER * bench.SOLVES_PER_ZONE
    assert r["flops_per_zone"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops * 1e6 / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / (152 * 128 * 2 * 2.070e9 / 1e12))
    assert r["hbm"]["achieved"] == pytest.approx(32 * 1e6 / 1e-3 / 1e9)
    assert r["bound"] == "alu" and r["traffic"] is None


def test_state_error_is_relative_per_field():
    rng = np.random.default_rng(0)
    b = rng.uniform(1.0, 2.0, (4, 8, 8))
    a = b.copy()
    a[2, 3, 4] += 1e-3
    tot = np.array([b[0].sum(), 0.0, 0.0, b[3].sum()])
    e = bench.state_error(a, b, tot, tot, tot)
    assert e["l1_rel"]["rho"] == 0.0 and e["max_rel"]["E"] == 0.0
    assert e["max_rel"]["rho_v"] == pytest.approx(1e-3 / np.abs(b[2]).max())
    assert e["l1_rel"]["rho_v"] == pytest.approx(1e-3 / np.abs(b[2]).sum())
    assert all(v == 0.0 for v in e["conservation_drift"].values())
