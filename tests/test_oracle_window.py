"""Pins of the differentiable-window oracle (oracle/window.py).

The oracle's forward is the hybrid step of the CPU oracle written again in
PyTorch; its gradient is autograd's. Pinned by: the forward against the C
oracle on the same inputs (fields, counters, particles), a closed form at
zero steps, and central finite differences of its own forward for every
kind of parameter (mode amplitudes, cosmic-ray drift, faux-shock kick).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as o  # noqa: E402
from oracle import window as wo  # noqa: E402
from tests import window_inputs as WI  # noqa: E402


def small_spec(nx=64, ppc=8, **kw):
    X, V = WI.plasma(nx, ppc)
    amps, ph = WI.modes()
    c = dict(WI.COMMON)
    c.update(kw)
    return wo.WindowSpec(nx=nx, ppc=ppc, X0=X, V0=V, phases=ph, **c), amps


def test_forward_matches_the_cpu_oracle():
    spec, amps = small_spec()
    th = WI.theta(amps)
    win = wo.Window(spec)
    with torch.no_grad():
        win.run(torch.tensor(th), 30)
        B0 = wo.Window(spec).initial_B(torch.tensor(amps)).numpy()
    sim = o.Oracle(dim=1, nx=spec.nx, ny=1, init_plasma=0, ppc=spec.ppc, cr_enable=1,
                   u_cr=WI.U_CR, u2=WI.U2, fs_mode_thermal=o.FS_SHOCK, p_iso=100.0,
                   n_cr_ratio=0.01, **WI.COMMON)
    X0 = spec.X0
    ci = np.floor(X0).astype(np.int32)
    z = np.zeros(len(X0))
    sim.inject(ci, z.astype(np.int32), X0 - ci, z, spec.V0[:, 0], spec.V0[:, 1],
               spec.V0[:, 2], ids=np.arange(len(X0), dtype=np.uint32))
    sim.set_B(B0)
    sim.step(30)
    d = sim.diag()
    for k in ("incident", "reflected", "transmitted", "escaped", "injected"):
        assert win.counts[k] == d[k], k
    assert d["reflected"] > 0 and d["injected"] > 0
    Bt = win.final["B"].numpy()
    assert np.abs(sim.grid(o.GRID_B)[0] - Bt).max() <= 1e-10 * np.abs(Bt).max()
    p = sim.particles()
    oid = np.argsort(p["id"])
    tid = np.argsort(win.final["ids"])
    assert np.array_equal(p["id"][oid].astype(np.int64), win.final["ids"][tid])
    assert np.array_equal(p["ci"][oid], win.final["ci"][tid])
    np.testing.assert_allclose(p["vx"][oid], win.final["V"].numpy()[tid, 0], rtol=1e-9,
                               atol=1e-9)


def test_zero_steps_closed_form():
    # modes m <= 16 are orthogonal on 64 cells: L = sum_m a_m^2 nx dx
    spec, amps = small_spec()
    L, g, _ = wo.loss_and_grad(spec, WI.theta(amps), 0)
    box = spec.nx * spec.dx
    assert L == pytest.approx(np.sum(amps ** 2) * box, rel=1e-12)
    np.testing.assert_allclose(g[:16], 2.0 * amps * box, rtol=1e-10)
    assert g[16] == 0.0 and g[17] == 0.0


@pytest.mark.parametrize("k", [0, 9, 16, 17])
def test_gradient_matches_central_differences(k):
    spec, amps = small_spec()
    th = WI.theta(amps)
    steps = 40
    L, g, win = wo.loss_and_grad(spec, th, steps)
    assert win.counts["reflected"] > 0
    h = 1e-6 * max(abs(th[k]), 1e-2)
    tp, tm = th.copy(), th.copy()
    tp[k] += h
    tm[k] -= h
    fd = (wo.loss_only(spec, tp, steps) - wo.loss_only(spec, tm, steps)) / (2 * h)
    assert g[k] == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(L)), (k, g[k], fd)
