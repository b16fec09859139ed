"""Differentiable window on the GPU: the CUDA forward and adjoint through the
C ABI (fs_window_*), against the FP64 PyTorch oracle (autograd) on a 64-cell,
8-ppc copy, and against central finite differences of the CUDA forward on
the full differentiable-window workload (2048 cells, 128 ppc, 200 steps
checkpointed every 20).
"""
import numpy as np
import pytest

from tests import window_inputs as WI

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_14282_gb300 import build
    build.build()
    from paper_2507_14282_gb300 import window as m
    return m


def gpu_window(fsw, nx, ppc, steps, ckpt, precision=0, loss_i0=0):
    X, V = WI.plasma(nx, ppc)
    amps, ph = WI.modes()
    w = fsw.FauxShockWindow(X, V, ph, steps=steps, ckpt=ckpt, loss_i0=loss_i0, nx=nx, ny=1,
                            ppc=ppc, precision=precision, cr_enable=1, fs_mode_thermal=1,
                            p_iso=100.0, n_cr_ratio=0.01, **WI.COMMON)
    return w, WI.theta(amps)


@pytest.fixture(scope="module")
def oracle_small():
    from oracle import window as wo
    X, V = WI.plasma(64, 8)
    amps, ph = WI.modes()
    spec = wo.WindowSpec(nx=64, ppc=8, X0=X, V0=V, phases=ph, **WI.COMMON)
    L, g, win = wo.loss_and_grad(spec, WI.theta(amps), 200)
    return L, g, win.counts


def test_fp64_forward_and_gradient_match_the_oracle_adjoint(fsw, oracle_small):
    L0, g0, counts0 = oracle_small
    w, th = gpu_window(fsw, 64, 8, 200, 20)
    L, g = w.loss_and_grad(th)
    c = w.counts()
    for k in ("incident", "reflected", "transmitted", "escaped", "injected"):
        assert c[k] == counts0[k], (k, c[k], counts0[k])
    assert c["reflected"] > 0 and c["injected"] > 0
    # every kind of parameter has a gradient well above round-off
    assert np.abs(g0[:16]).min() > 1e-3 and abs(g0[16]) > 1e-5 and abs(g0[17]) > 1e-3
    assert L == pytest.approx(L0, rel=1e-9)
    # modes (scale: their largest gradient), then u_cr and u2 each on its own
    gm = np.abs(g0[:16]).max()
    np.testing.assert_allclose(g[:16], g0[:16], rtol=0, atol=1e-6 * gm)
    assert g[16] == pytest.approx(g0[16], rel=1e-5)
    assert g[17] == pytest.approx(g0[17], rel=1e-6)
    w.close()


def test_checkpoint_interval_does_not_change_the_gradient(fsw):
    w1, th = gpu_window(fsw, 64, 8, 60, 20)
    w2, _ = gpu_window(fsw, 64, 8, 60, 60)
    w3, _ = gpu_window(fsw, 64, 8, 60, 7)
    L1, g1 = w1.loss_and_grad(th)
    L2, g2 = w2.loss_and_grad(th)
    L3, g3 = w3.loss_and_grad(th)
    assert L1 == L2 == L3
    np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(g3, g1, rtol=1e-12, atol=1e-15)
    # a second forward gives the same loss (the window keeps its inputs)
    assert w1.forward(th) == L1


def test_autograd_function_runs_the_cuda_adjoint(fsw):
    import torch
    w, th = gpu_window(fsw, 64, 8, 40, 20)
    t = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    loss = fsw.window_loss(w, t)
    (3.0 * loss).backward()
    L, g = w.loss_and_grad(th)
    assert float(loss.detach()) == L
    np.testing.assert_allclose(t.grad.numpy(), 3.0 * g, rtol=1e-12, atol=1e-18)


@pytest.fixture(scope="module")
def full_fp64(fsw):
    w, th = gpu_window(fsw, 2048, 128, 200, 20)
    L, g = w.loss_and_grad(th)
    return w, th, L, g


@pytest.fixture(scope="module")
def full_fp64_100(fsw):
    w, th = gpu_window(fsw, 2048, 128, 100, 20)
    L, g = w.loss_and_grad(th)
    return w, th, L, g


def central_difference(w, th, k, L, rel_h):
    h = rel_h * max(abs(th[k]), 1e-2)
    tp, tm = th.copy(), th.copy()
    tp[k] += h
    tm[k] -= h
    fd = (w.forward(tp) - w.forward(tm)) / (2 * h)
    # far above what FP64 rounding of the loss can give over 2 h
    assert abs(fd) > 1e-12 * abs(L) / h
    return fd


# The loss is piecewise differentiable: CIC weights have kinks where a
# particle crosses a cell face, and a returned ion's re-placement and path
# move with u2 and u_cr. A difference interval must be narrower than the
# spacing of the kinks it crosses and wider than rounding: for the kick u2
# that is h = 1e-6 u2 (1e-4 straddles kinks and moves the quotient by 2 %,
# 1e-5 by 0.4 %); the modes take h = 1e-5 |a_m| (an h sweep from 1e-4 to
# 1e-6 |a_m| on GB300 gave agreement within 2e-5 for every mode).
@pytest.mark.parametrize("k,rel_h", [(m, 1e-5) for m in range(16)] + [(17, 1e-6)])
def test_full_window_gradient_matches_central_differences(full_fp64, k, rel_h):
    w, th, L, g = full_fp64
    fd = central_difference(w, th, k, L, rel_h)
    assert g[k] == pytest.approx(fd, rel=1e-3), (k, g[k], fd)


def test_cosmic_ray_drift_gradient_matches_central_differences(full_fp64_100, full_fp64):
    # d L / d u_cr is 1e7 times smaller than the mode gradients; over 100
    # steps the difference quotient converges and agrees with the adjoint to
    # 1e-3. Over 200 steps the kinks of thousands of cosmic-ray crossings make
    # the quotient wander by about 1 % across a decade of h around the
    # adjoint's value.
    w, th, L, g = full_fp64_100
    fd = central_difference(w, th, 16, L, 1e-6)
    assert g[16] == pytest.approx(fd, rel=1e-3), (g[16], fd)
    # 200 steps, h swept over 1e-6 and 1e-7 |u_cr| (a sweep from 1e-4 down
    # on GB300 gave quotients from -4.5 % to +0.8 % of the adjoint): each
    # quotient within 2 % and the adjoint between them
    w, th, L, g = full_fp64
    fds = [central_difference(w, th, 16, L, rh) for rh in (1e-6, 1e-7)]
    for fd in fds:
        assert g[16] == pytest.approx(fd, rel=2e-2), (g[16], fds)
    assert min(fds) <= g[16] <= max(fds), (g[16], fds)


def test_fp32_window_gradient_tracks_fp64(fsw, full_fp64):
    # the full window (200 steps): the FP32 forward makes one faux-shock
    # return decision differently from the FP64 run (893 against 891 returns)
    # and its gradient follows its own trajectory: modes within 1e-3 of the
    # FP64 gradient (2.7e-4 on GB300), the kick within 2 % (0.7 %)
    _, th, L64, g64 = full_fp64
    w, _ = gpu_window(fsw, 2048, 128, 200, 20, precision=1)
    L32, g32 = w.loss_and_grad(th)
    assert L32 == pytest.approx(L64, rel=1e-3)
    gm = np.abs(g64[:16]).max()
    assert np.abs(g32[:16] - g64[:16]).max() <= 1e-3 * gm
    assert g32[17] == pytest.approx(g64[17], rel=2e-2)
    w.close()


def test_fp32_window_gradient_equals_fp64_while_the_decisions_agree(fsw):
    # over 20 steps both forwards take the same faux-shock decisions (counts
    # equal): the FP32 adjoint then gives the FP64 gradient to 1e-4 in every
    # component (about 1e-8 for the modes and 1e-5 for u_cr and u2 on GB300)
    w64, th = gpu_window(fsw, 2048, 128, 20, 20, precision=0)
    w32, _ = gpu_window(fsw, 2048, 128, 20, 20, precision=1)
    L64, g64 = w64.loss_and_grad(th)
    L32, g32 = w32.loss_and_grad(th)
    assert w32.counts() == w64.counts()
    assert L32 == pytest.approx(L64, rel=1e-6)
    gm = np.abs(g64[:16]).max()
    assert np.abs(g32[:16] - g64[:16]).max() <= 1e-4 * gm
    assert g32[16] == pytest.approx(g64[16], rel=1e-4)
    assert g32[17] == pytest.approx(g64[17], rel=1e-4)
    w64.close()
    w32.close()


@pytest.mark.parametrize("nx,n_sub", [(40, 2), (72, 1), (88, 3)])
def test_ragged_tiles_and_substeps_match_the_oracle(fsw, nx, n_sub):
    """The field kernels work on 16-cell tiles with halos of 4 n_sub + 2
    (forward) and 8 n_sub + 3 (reverse) cells: grids that end in a partial
    tile, with one to three RK4 substeps per step, against the oracle."""
    from oracle import window as wo
    X, V = WI.plasma(nx, 8)
    amps, ph = WI.modes()
    th = WI.theta(amps)
    spec = wo.WindowSpec(nx=nx, ppc=8, X0=X, V0=V, phases=ph, n_sub=n_sub, **WI.COMMON)
    L0, g0, win = wo.loss_and_grad(spec, th, 100)
    w = fsw.FauxShockWindow(X, V, ph, steps=100, ckpt=20, nx=nx, ny=1, ppc=8, n_sub=n_sub,
                            precision=0, cr_enable=1, fs_mode_thermal=1, p_iso=100.0,
                            n_cr_ratio=0.01, **WI.COMMON)
    L, g = w.loss_and_grad(th)
    assert w.counts() == win.counts
    assert L == pytest.approx(L0, rel=1e-9)
    gm = np.abs(g0[:16]).max()
    np.testing.assert_allclose(g[:16], g0[:16], rtol=0, atol=1e-6 * gm)
    assert g[16] == pytest.approx(g0[16], rel=1e-5)
    assert g[17] == pytest.approx(g0[17], rel=1e-6)
    # the FP32 window on the same ragged grid tracks it
    w32 = fsw.FauxShockWindow(X, V, ph, steps=100, ckpt=20, nx=nx, ny=1, ppc=8, n_sub=n_sub,
                              precision=1, cr_enable=1, fs_mode_thermal=1, p_iso=100.0,
                              n_cr_ratio=0.01, **WI.COMMON)
    L32, g32 = w32.loss_and_grad(th)
    assert L32 == pytest.approx(L0, rel=1e-3)
    assert np.abs(g32[:16] - g0[:16]).max() <= 2e-2 * gm
