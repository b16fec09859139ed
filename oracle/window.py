"""TEST INFRASTRUCTURE ONLY: the differentiable window of the 1D faux-shock
box written in plain PyTorch (CPU, float64) and differentiated by autograd.

This is the oracle for the adjoint (the gradient of a loss at the end of a
window of steps with respect to seeded B modes, the cosmic-ray drift speed
and the faux-shock kick). It takes the hybrid step in the order of the
scheme (Sec. 2: kinetic ions, massless isothermal electrons, the faux shock
at x = 0 of Eq. 1, inflow at x = L and the cosmic-ray source at the faux
shock), one step at a time:

  1. gather E, Bbar at the particle (CIC, two nodes);
  2. Boris push (non-relativistic);
  3. move; open far wall (removed); faux shock at x = 0: the return
     decision U0 < P(v) (Eq. 1) is a branch, the returned velocity
     (downstream-frame speed kept, flux-weighted direction, boost back by
     u2) and the re-placement are differentiable;
  4. injection: thermal plasma at x = L, cosmic rays at x = 0 with speed
     p_iso, flux-weighted in the frame drifting at u_cr;
  5. deposit n, J at nodes (CIC), wall nodes x2, density floor, u = J/n;
  6. RK4 substeps of dB/dt = -curl E(B) with n, u frozen; then E and Bbar.

Branches (which particles cross, are returned, escape, which node they sit
next to, the density floor) are taken from the forward values and are not
differentiated: gradients are those of the discrete map with the branches
frozen. Random draws come from the CPU oracle's own Philox, log and sincos
(pinned in its tests), keyed on particle number and step exactly as in the
oracle's step. The only library routines are PyTorch tensor arithmetic and
autograd; nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from oracle import oracle as o

PURPOSE_FS, PURPOSE_INJ_A, PURPOSE_INJ_B, PURPOSE_INJ_CR = 3, 4, 5, 6
OFFMAX = 1.0 - 2.0 ** -53
TD = torch.float64


@dataclass
class WindowSpec:
    """A 1D faux-shock box (canonical frame: faux shock at x = 0, inflow at
    x = L moving in -x). Positions of the initial particles in cells
    (X = i + f), velocities in v_A; mode phases phi_m of the seeded
    transverse B modes; the loss sums |B_perp - B0_perp|^2 dx over the
    cells i >= loss_i0."""
    nx: int
    dx: float
    dt: float
    mach_a: float
    theta_bn_deg: float
    beta_i: float
    beta_e: float
    ppc: int
    seed: int
    X0: np.ndarray
    V0: np.ndarray
    phases: np.ndarray
    loss_i0: int = 0
    n_sub: int = 2
    n_floor: float = 0.05
    fs_mode_thermal: int = 1       # 1: the faux shock returns thermal ions too
    fs_frame: int = 0              # speed of Eq. 1 in the shock frame
    cr_enable: int = 1
    inject_thermal: int = 1
    n_cr_ratio: float = 0.01
    p_iso: float = 100.0
    ids0: np.ndarray = field(default=None)

    @property
    def nxn(self):
        return self.nx + 1


def draw4(seed: int, pid: int, step: int, purpose: int) -> np.ndarray:
    return o.philox([pid, step & 0xFFFFFFFF, purpose, 0],
                    [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])


def gauss2(u1: float, u2: float):
    rad = math.sqrt(-2.0 * o.log(u1))
    c, s = o.sincos2pi(u2)
    return rad * c, rad * s


class Window:
    """One forward pass of the window; loss() is differentiable in theta =
    (a_1 .. a_M, u_cr, u2)."""

    def __init__(self, spec: WindowSpec):
        self.s = spec
        th = math.radians(spec.theta_bn_deg)
        self.b0 = (math.cos(th), math.sin(th), 0.0)
        self.te = 0.5 * spec.beta_e
        self.vth = math.sqrt(0.5 * spec.beta_i)
        self.dtdx = spec.dt / spec.dx
        self.hdt = 0.5 * spec.dt
        self.idx = 1.0 / spec.dx
        self.hdx = 0.5 / spec.dx
        self.h = spec.dt / spec.n_sub
        self.w_th = 1.0 / spec.ppc
        self.w_cr = spec.n_cr_ratio / spec.ppc
        self.rate = spec.ppc * spec.mach_a * spec.dt / spec.dx
        self.counts = dict(incident=0, reflected=0, transmitted=0, escaped=0, injected=0)

    # ------------------------------------------------------------ fields
    def initial_B(self, amps):
        s = self.s
        x = (torch.arange(s.nx, dtype=TD) + 0.5) * s.dx
        L = s.nx * s.dx
        ph = torch.as_tensor(s.phases, dtype=TD)
        m = torch.arange(1, len(s.phases) + 1, dtype=TD)
        arg = 2.0 * math.pi * m[:, None] * x[None, :] / L + ph[:, None]
        by = self.b0[1] + (amps[:, None] * torch.cos(arg)).sum(0)
        bz = self.b0[2] + (amps[:, None] * torch.sin(arg)).sum(0)
        bx = torch.full((s.nx,), self.b0[0], dtype=TD)
        return torch.stack([bx, by, bz], 1)  # [nx][3]

    def ohm(self, B, n, u):
        """E and Bbar at the nx + 1 nodes; zero-gradient ghost cells at the
        walls, mirrored density gradient."""
        s = self.s
        i = np.arange(s.nxn)
        im = np.clip(i - 1, 0, s.nx - 1)
        ip = np.clip(i, 0, s.nx - 1)
        Bm, Bp = B[im], B[ip]
        bb = 0.5 * (Bm + Bp)
        dby = (Bp[:, 1] - Bm[:, 1]) * self.idx
        dbz = (Bp[:, 2] - Bm[:, 2]) * self.idx
        ax = torch.zeros_like(dby)
        ay, az = -dbz, dby
        ipn = i + 1
        ipn = np.where(ipn > s.nx, 2 * s.nx - ipn, ipn)
        imn = np.abs(i - 1)
        dnx = (n[ipn] - n[imn]) * self.hdx
        bbx, bby, bbz = bb[:, 0], bb[:, 1], bb[:, 2]
        ux, uy, uz = u[:, 0], u[:, 1], u[:, 2]
        cax = ay * bbz - az * bby
        cay = az * bbx - ax * bbz
        caz = ax * bby - ay * bbx
        cux = uy * bbz - uz * bby
        cuy = uz * bbx - ux * bbz
        cuz = ux * bby - uy * bbx
        ex = (-(self.te * dnx) + cax) / n - cux
        ey = cay / n - cuy
        ez = caz / n - cuz
        return torch.stack([ex, ey, ez], 1), bb

    def curl_K(self, E):
        """-curl E at the cell centres (1D: dB_y/dt = dE_z/dx, dB_z/dt = -dE_y/dx)."""
        dez = (E[1:, 2] - E[:-1, 2]) * self.idx
        dey = (E[1:, 1] - E[:-1, 1]) * self.idx
        return torch.stack([torch.zeros_like(dez), dez, -dey], 1)

    def advance(self, B, n, u):
        h, hh, h6 = self.h, 0.5 * self.h, self.h / 6.0
        for _ in range(self.s.n_sub):
            k1 = self.curl_K(self.ohm(B, n, u)[0])
            k2 = self.curl_K(self.ohm(B + hh * k1, n, u)[0])
            k3 = self.curl_K(self.ohm(B + hh * k2, n, u)[0])
            k4 = self.curl_K(self.ohm(B + h * k3, n, u)[0])
            B = B + h6 * (((k1 + 2.0 * k2) + 2.0 * k3) + k4)
        return B

    # ------------------------------------------------------------ moments
    def deposit(self, ci, f, V, W):
        s = self.s
        nr = torch.zeros(s.nxn, dtype=TD)
        J = torch.zeros(s.nxn, 3, dtype=TD)
        i0 = torch.as_tensor(ci, dtype=torch.long)
        c0 = W * (1.0 - f)
        c1 = W * f
        nr = nr.index_add(0, i0, c0).index_add(0, i0 + 1, c1)
        J = J.index_add(0, i0, c0[:, None] * V).index_add(0, i0 + 1, c1[:, None] * V)
        wall = torch.ones(s.nxn, dtype=TD)
        wall[0] = wall[-1] = 2.0
        nr = nr * wall
        J = J * wall[:, None]
        n = torch.where(nr.detach() < s.n_floor, torch.full_like(nr, s.n_floor), nr)
        return n, J / n[:, None]

    # ------------------------------------------------------------ particles
    @staticmethod
    def boris(V, E, B, hdt):
        em = hdt * E
        vm = V + em
        t = hdt * B
        tt = (t * t).sum(1, keepdim=True)
        fct = 2.0 / (1.0 + tt)
        sv = fct * t
        p = vm + torch.cross(vm, t, dim=1)
        q = vm + torch.cross(p, sv, dim=1)
        return q + em

    def run(self, theta: torch.Tensor, steps: int):
        """Loss after `steps` steps; theta = (a_1..a_M, u_cr, u2) float64."""
        s = self.s
        M = len(s.phases)
        amps, u_cr, u2 = theta[:M], theta[M], theta[M + 1]
        u2v = float(u2.detach())
        fsp = o.make_params(u2=u2v, fs_speed_frame=s.fs_frame, seed=s.seed)
        # particle state: integer cell (numpy) and differentiable offset
        X0 = np.asarray(s.X0, np.float64)
        ci = np.floor(X0).astype(np.int64)
        f = torch.as_tensor(X0 - ci, dtype=TD)
        V = torch.as_tensor(np.asarray(s.V0, np.float64), dtype=TD)
        ids = (np.arange(len(X0), dtype=np.int64) if s.ids0 is None
               else np.asarray(s.ids0, np.int64))
        W = torch.full((len(X0),), self.w_th, dtype=TD)
        cr = np.zeros(len(X0), bool)
        next_id = int(ids.max()) + 1 if len(ids) else 0
        acc = 0.0
        B = self.initial_B(amps)
        n, u = self.deposit(ci, f, V, W)
        E, Bb = self.ohm(B, n, u)
        for step in range(steps):
            # 1-2: gather and push
            Ep = (1.0 - f)[:, None] * E[ci] + f[:, None] * E[ci + 1]
            Bp = (1.0 - f)[:, None] * Bb[ci] + f[:, None] * Bb[ci + 1]
            V = self.boris(V, Ep, Bp, self.hdt)
            # 3: move and walls
            fr = f + V[:, 0] * self.dtdx
            k = np.floor(fr.detach().numpy()).astype(np.int64)
            inew = ci + k
            fn = fr - torch.as_tensor(k, dtype=TD)
            fn = torch.where(fn.detach() >= 1.0, torch.full_like(fn, OFFMAX), fn)
            keep = np.ones(len(ci), bool)
            newV = [V[q] for q in range(len(ci))]
            newf = [fn[q] for q in range(len(ci))]
            for q in np.nonzero(inew >= s.nx)[0]:
                keep[q] = False
                self.counts["escaped"] += 1
            for q in np.nonzero(inew < 0)[0]:
                self.counts["incident"] += 1
                mode = 1 if cr[q] else s.fs_mode_thermal
                v = V[q].detach().numpy().copy()
                ret = False
                if mode == 1:
                    ret, _, _ = o.fs_rule(v, int(ids[q]) & o.ID_MASK, step, u2=u2v,
                                          fs_speed_frame=s.fs_frame, seed=s.seed)
                if not ret:
                    keep[q] = False
                    self.counts["transmitted"] += 1
                    continue
                self.counts["reflected"] += 1
                r = draw4(s.seed, int(ids[q]) & o.ID_MASK, step, PURPOSE_FS)
                U1, U2 = o.u01(int(r[1])), o.u01(int(r[2]))
                c, sn2 = o.sincos2pi(U2)
                vx, vy, vz = V[q, 0], V[q, 1], V[q, 2]
                wx = vx + u2
                w = torch.sqrt(wx * wx + vy * vy + vz * vz)
                a = u2 / w
                mu = a + (1.0 - a) * math.sqrt(U1)
                snm = torch.sqrt(1.0 - mu * mu)
                vnew = torch.stack([w * mu - u2, w * snm * c, w * snm * sn2])
                Xo = ci[q] + f[q]
                Xn = ci[q] + fr[q]
                g = Xn / (Xn - Xo)
                fq = g * (vnew[0] * self.dtdx)
                if float(fq.detach()) < 0.0:
                    fq = torch.zeros((), dtype=TD)
                elif float(fq.detach()) >= 1.0:
                    fq = torch.full((), OFFMAX, dtype=TD)
                newV[q] = vnew
                newf[q] = fq
                inew[q] = 0
                ids[q] |= o.ID_RETURNED
            sel = np.nonzero(keep)[0]
            ci = inew[sel]
            f = torch.stack([newf[q] for q in sel]) if len(sel) else fn[:0]
            V = torch.stack([newV[q] for q in sel]) if len(sel) else V[:0]
            W = W[torch.as_tensor(sel, dtype=torch.long)]
            cr = cr[sel]
            ids = ids[sel]
            # 4: injection (thermal at x = L, then cosmic rays at x = 0)
            acc = acc + self.rate
            fl = math.floor(acc)
            nnew = int(fl)
            acc = acc - fl
            add_ci, add_f, add_V, add_W, add_cr, add_id = [], [], [], [], [], []
            if s.inject_thermal:
                for _ in range(nnew):
                    pid = next_id
                    next_id += 1
                    ra = draw4(s.seed, pid, step, PURPOSE_INJ_A)
                    rb = draw4(s.seed, pid, step, PURPOSE_INJ_B)
                    g0, g1 = gauss2(o.u01(int(ra[0])), o.u01(int(ra[1])))
                    g2, _ = gauss2(o.u01(int(ra[2])), o.u01(int(ra[3])))
                    vx = self.vth * g0 - s.mach_a
                    X = float(s.nx) - (o.u01(int(rb[0])) * abs(vx)) * self.dtdx
                    i = int(math.floor(X))
                    fx = X - math.floor(X)
                    if i >= s.nx:
                        i, fx = s.nx - 1, OFFMAX
                    if i < 0:
                        i, fx = 0, 0.0
                    if fx >= 1.0:
                        fx = OFFMAX
                    add_ci.append(i)
                    add_f.append(torch.tensor(fx, dtype=TD))
                    add_V.append(torch.tensor([vx, self.vth * g1, self.vth * g2], dtype=TD))
                    add_W.append(self.w_th)
                    add_cr.append(False)
                    add_id.append(pid)
                    self.counts["injected"] += 1
            if s.cr_enable:
                for _ in range(nnew):
                    pid = next_id
                    next_id += 1
                    rc = draw4(s.seed, pid, step, PURPOSE_INJ_CR)
                    a = u_cr / s.p_iso
                    mu = a + (1.0 - a) * math.sqrt(o.u01(int(rc[0])))
                    snm = torch.sqrt(1.0 - mu * mu)
                    c, sn2 = o.sincos2pi(o.u01(int(rc[1])))
                    vx = s.p_iso * mu - u_cr
                    Vn = torch.stack([vx, s.p_iso * snm * c, s.p_iso * snm * sn2])
                    X = (o.u01(int(rc[2])) * vx) * self.dtdx
                    i = int(math.floor(float(X.detach())))
                    fx = X - float(i)
                    if i >= s.nx:
                        i, fx = s.nx - 1, torch.tensor(OFFMAX, dtype=TD)
                    if i < 0:
                        i, fx = 0, torch.tensor(0.0, dtype=TD)
                    if float(fx.detach()) >= 1.0:
                        fx = torch.tensor(OFFMAX, dtype=TD)
                    add_ci.append(i)
                    add_f.append(fx)
                    add_V.append(Vn)
                    add_W.append(self.w_cr)
                    add_cr.append(True)
                    add_id.append(pid | o.ID_CR)
                    self.counts["injected"] += 1
            if add_ci:
                ci = np.concatenate([ci, np.array(add_ci, np.int64)])
                f = torch.cat([f, torch.stack(add_f)])
                V = torch.cat([V, torch.stack(add_V)])
                W = torch.cat([W, torch.tensor(add_W, dtype=TD)])
                cr = np.concatenate([cr, np.array(add_cr, bool)])
                ids = np.concatenate([ids, np.array(add_id, np.int64)])
            # 5-6: moments and fields
            n, u = self.deposit(ci, f, V, W)
            B = self.advance(B, n, u)
            E, Bb = self.ohm(B, n, u)
        self.final = dict(B=B, ci=ci, f=f, V=V, ids=ids, n=n, u=u, E=E)
        d = B[s.loss_i0:, 1:] - torch.tensor(self.b0[1:], dtype=TD)
        return (d * d).sum() * s.dx


def loss_and_grad(spec: WindowSpec, theta, steps: int):
    """(loss, d loss / d theta, the window) with the branches frozen."""
    th = torch.tensor(np.asarray(theta, np.float64), dtype=TD, requires_grad=True)
    win = Window(spec)
    L = win.run(th, steps)
    L.backward()
    return float(L.detach()), th.grad.numpy().copy(), win


def loss_only(spec: WindowSpec, theta, steps: int) -> float:
    with torch.no_grad():
        return float(Window(spec).run(torch.tensor(np.asarray(theta, np.float64), dtype=TD),
                                      steps))
