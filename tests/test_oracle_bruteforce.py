"""Brute force: the whole substep re-derived in plain numpy on an 8x8 grid,
written from the paper's printed equations and the stated readings, not from
the oracle, and compared with the oracle to 1e-12.

- step 1 (Sec. 2.1): MinMod-limited J and f = H/J at each face (|f| scaled to
  1), the printed Levermore closure, the corrected GLF J flux with eps(tau) and
  the diffusion term, the modified GLF K flux, donor-cell advection with the
  face velocity, the work term -grad u : K / c from the cell's own closure;
- step 2: the closed rearrangement of the implicit emission/absorption step;
- the force 4 pi / (c c_tilde dt) sum_k dnu_k (H' - H'') (Sec. 2.3);
- step 3 (App. A): <H>_k from the printed I(x, a) (scipy's erf and Dawson),
  K_k and C_k with the recoil factor and the Doppler term, the leakage
  coefficients in the printed phi / chi form assembled into a dense matrix and
  solved with numpy.linalg.solve (BDF1, zero-flux ends; |P| kept below the
  printed form's overflow, which the oracle's rearranged form avoids), then
  H = (J'''/J'') H'' and the causality cap.
A dropped term, a wrong sign or a transposed index in either implementation
shows up as a mismatch far above 1e-12.
"""
import math

import numpy as np
import pytest
from scipy import special as sp

import oracle

C = 2.99792458e10
KB, HPL, MH = 1.380649e-16, 6.62607015e-27, 1.67353284e-24
ME, QE = 9.1093837015e-28, 4.803204712570263e-10
NU0 = C / 1215.67e-8
A_LYA, F12 = 6.265e8, 0.4162


def line(T):
    dnuD = NU0 * math.sqrt(2.0 * KB * T / MH) / C
    a = A_LYA / (4.0 * math.pi * dnuD)
    sigma0 = math.sqrt(math.pi) * QE * QE * F12 / (ME * C * dnuD)
    return dnuD, a, sigma0


def I_voigt(x, a):
    # App. A: I(x, a) = sqrt(pi)/2 erf(x) - (2a/sqrt(pi)) F(x) + a^2 x exp(-x^2)
    return (math.sqrt(math.pi) / 2.0) * sp.erf(x) - (2.0 * a / math.sqrt(math.pi)) * sp.dawsn(x) \
        + a * a * x * np.exp(-x * x)


def closure(fx, fy):
    f2 = fx * fx + fy * fy
    chi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * math.sqrt(4.0 - 3.0 * f2))
    a = (1.0 - chi) / 2.0
    if f2 == 0.0:
        return a, 0.0, a, a  # Dxx, Dxy, Dyy, Dphiphi
    b = (3.0 * chi - 1.0) / 2.0 / f2
    return a + b * fx * fx, b * fx * fy, a + b * fy * fy, a


def cap(fx, fy):
    f = math.hypot(fx, fy)
    return (fx / f, fy / f) if f > 1.0 else (fx, fy)


def minmod(a, b):
    if a * b <= 0.0:
        return 0.0
    return a if abs(a) < abs(b) else b


def prim(J, H1, H2):
    return (H1 / J, H2 / J) if J > 0.0 else (0.0, 0.0)


def brute_substep(p, J, Hx, Hy, bands=None, prune=0.0, diag=None):
    """bands: (alpha_F, kappa, j) per [band][cell] for broad bands (Sec. 3):
    each band is one frequency-integrated group (dnu = 1) with the given flux
    and absorption opacities and emissivity, and no step 3.  prune: bins
    holding no more than this share of sum_k dnu_k sum_cells J_k skip step 1
    (Sec. 2.2).  diag: a dict that receives the J face fluxes, the work term,
    kappa, j and J'' of every bin, with c_tilde dt and the bin widths."""
    nx, ny, dx = p["nx"], p["ny"], p["dx"]
    if bands is None:
        e = p["edges"]
        nb = e.size - 1
        dnu = np.diff(e)
        nubar = NU0 + 0.5 * (e[1:] + e[:-1])
    else:
        nb = bands[0].shape[0]
        dnu = np.ones(nb)
    # per-cell line constants and tables (App. A at each cell's own temperature)
    Tc = p.get("temp")
    Tc = np.full((ny, nx), p["T"]) if Tc is None else Tc
    Hkc = np.zeros((nb, ny, nx))
    wc = np.zeros((nb, ny, nx))
    dnuDc = np.empty((ny, nx))
    s0c = np.zeros((ny, nx))
    for j in range(ny if bands is None else 0):
        for i in range(nx):
            dD, av, s0 = line(Tc[j, i])
            xx = e / dD
            h = (I_voigt(xx[1:], av) - I_voigt(xx[:-1], av)) / (dnu / dD)
            ww = h * (dnu / dD)
            Hkc[:, j, i] = h
            wc[:, j, i] = ww / ww.sum()
            dnuDc[j, i] = dD
            s0c[j, i] = s0
    alpha = p["n_hi"] * s0c
    rho, pd, ux, uy, lum = p["rho_d"], p["p_d"], p["ux"], p["uy"], p["lum"]
    kabs, kF = p["kappa_abs"], p["kappa_F"]
    ct = p["c_tilde"]
    umax = np.hypot(ux, uy).max()
    dt = (p["cfl"] / 2.0) * dx / (ct + umax)
    cdt = ct * dt
    bc = p["bc"]
    V = dx ** 3

    def clampi(i, n):
        return min(max(i, 0), n - 1)

    # velocity gradients: central differences, ghost = edge cell
    gxx = np.zeros((ny, nx))
    gyy = np.zeros((ny, nx))
    gsh = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            xm, xp = clampi(i - 1, nx), clampi(i + 1, nx)
            ym, yp = clampi(j - 1, ny), clampi(j + 1, ny)
            gxx[j, i] = (ux[j, xp] - ux[j, xm]) / (2 * dx)
            gyy[j, i] = (uy[yp, i] - uy[ym, i]) / (2 * dx)
            gsh[j, i] = (ux[yp, i] - ux[ym, i]) / (2 * dx) + (uy[j, xp] - uy[j, xm]) / (2 * dx)

    J1 = np.empty_like(J)
    Hx1 = np.empty_like(J)
    Hy1 = np.empty_like(J)
    W = np.zeros((nb, ny, nx))
    FXJk = np.zeros((nb, ny, nx + 1))
    FYJk = np.zeros((nb, ny + 1, nx))
    Ek = dnu * J.sum(axis=(1, 2))
    on = Ek > prune * Ek.sum() if prune > 0.0 else np.ones(nb, bool)
    for k in range(nb):
        if not on[k]:  # a pruned bin keeps its state through step 1
            J1[k], Hx1[k], Hy1[k] = J[k], Hx[k], Hy[k]
            continue
        aF = alpha * Hkc[k] + rho * kF if bands is None else bands[0][k]

        def cell(i, j, axis):
            # the state of a (possibly ghost) cell: (J, f_n, f_t), u_n, alpha_F
            n = nx if axis == 0 else ny
            idx = i if axis == 0 else j
            lo_side, hi_side = (0, 1) if axis == 0 else (2, 3)
            vac = (idx < 0 and bc[lo_side] == 1) or (idx >= n and bc[hi_side] == 1)
            ii, jj = (clampi(i, nx), j) if axis == 0 else (i, clampi(j, ny))
            u = ux[jj, ii] if axis == 0 else uy[jj, ii]
            if vac:
                return (0.0, 0.0, 0.0), u, aF[jj, ii]
            jv, h1, h2 = J[k, jj, ii], Hx[k, jj, ii], Hy[k, jj, ii]
            fx, fy = prim(jv, h1, h2)
            fn, ft = (fx, fy) if axis == 0 else (fy, fx)
            return (jv, fn, ft), u, aF[jj, ii]

        def face(q, u0, u1, a0, a1):
            # q: states of cells -1, 0, +1, +2 around the face between 0 and +1
            (Jm, nm, tm), (J0, n0, t0), (Jp, n1, t1), (J2, n2, t2) = q
            JL = J0 + 0.5 * minmod(J0 - Jm, Jp - J0)
            JR = Jp - 0.5 * minmod(Jp - J0, J2 - Jp)
            nL = n0 + 0.5 * minmod(n0 - nm, n1 - n0)
            tL = t0 + 0.5 * minmod(t0 - tm, t1 - t0)
            nR = n1 - 0.5 * minmod(n1 - n0, n2 - n1)
            tR = t1 - 0.5 * minmod(t1 - t0, t2 - t1)
            nL, tL = cap(nL, tL)
            nR, tR = cap(nR, tR)
            HnL, HtL, HnR, HtR = JL * nL, JL * tL, JR * nR, JR * tR
            DnnL, DntL, _, _ = closure(nL, tL)
            DnnR, DntR, _, _ = closure(nR, tR)
            tau = a0 * dx / 2.0 + a1 * dx / 2.0
            eps = (0.2 + tau) / (0.2 + tau + tau * tau)
            diff = (1.0 - eps) * (Jp - J0) / (3.0 * tau) if tau > 0.0 else 0.0
            wf = 0.5 * (u0 + u1) / C
            up = wf > 0.0
            FJ = eps * 0.5 * (HnL + HnR) - eps * 0.5 * (JR - JL) - diff + wf * (JL if up else JR)
            FN = 0.5 * (DnnL * JL + DnnR * JR) - eps * 0.5 * (HnR - HnL) + wf * (HnL if up else HnR)
            FT = 0.5 * (DntL * JL + DntR * JR) - eps * 0.5 * (HtR - HtL) + wf * (HtL if up else HtR)
            return FJ, FN, FT

        FXJ = np.zeros((ny, nx + 1))
        FXN = np.zeros((ny, nx + 1))
        FXT = np.zeros((ny, nx + 1))
        for j in range(ny):
            for i in range(nx + 1):  # face between cells i-1 and i
                cs = [cell(i - 2 + m, j, 0) for m in range(4)]
                FXJ[j, i], FXN[j, i], FXT[j, i] = face([c[0] for c in cs], cs[1][1], cs[2][1],
                                                       cs[1][2], cs[2][2])
        FYJ = np.zeros((ny + 1, nx))
        FYN = np.zeros((ny + 1, nx))
        FYT = np.zeros((ny + 1, nx))
        for j in range(ny + 1):
            for i in range(nx):
                cs = [cell(i, j - 2 + m, 1) for m in range(4)]
                FYJ[j, i], FYN[j, i], FYT[j, i] = face([c[0] for c in cs], cs[1][1], cs[2][1],
                                                       cs[1][2], cs[2][2])
        FXJk[k], FYJk[k] = FXJ, FYJ
        for j in range(ny):
            for i in range(nx):
                jv = J[k, j, i]
                fx, fy = cap(*prim(jv, Hx[k, j, i], Hy[k, j, i]))
                Dxx, Dxy, Dyy, _ = closure(fx, fy)
                W[k, j, i] = (Dxx * gxx[j, i] + Dyy * gyy[j, i] + Dxy * gsh[j, i]) * jv
                divJ = (FXJ[j, i + 1] - FXJ[j, i]) + (FYJ[j + 1, i] - FYJ[j, i])
                divHx = (FXN[j, i + 1] - FXN[j, i]) + (FYT[j + 1, i] - FYT[j, i])
                divHy = (FXT[j, i + 1] - FXT[j, i]) + (FYN[j + 1, i] - FYN[j, i])
                J1[k, j, i] = jv - cdt * (divJ / dx + W[k, j, i] / C)
                Hx1[k, j, i] = Hx[k, j, i] - cdt * divHx / dx
                Hy1[k, j, i] = Hy[k, j, i] - cdt * divHy / dx

    # step 2 and the force
    aH = alpha[None] * Hkc
    kap = rho[None] * kabs + pd[None] * aH
    aFk = aH + rho[None] * kF
    js = lum[None] * wc / (4.0 * math.pi * V * dnu[:, None, None])
    if bands is not None:
        aFk, kap, js = bands
    J2 = (J1 + cdt * js) / (1.0 + cdt * kap)
    Hx2 = Hx1 / (1.0 + cdt * aFk)
    Hy2 = Hy1 / (1.0 + cdt * aFk)
    fcoef = 4.0 * math.pi / (C * ct * dt)
    fx_out = fcoef * (dnu[:, None, None] * (Hx1 - Hx2)).sum(axis=0)
    fy_out = fcoef * (dnu[:, None, None] * (Hy1 - Hy2)).sum(axis=0)
    if diag is not None:
        shape = (nb, ny, nx)
        diag.update(FXJ=FXJk, FYJ=FYJk, W=W, kap=np.broadcast_to(kap, shape),
                    js=np.broadcast_to(js, shape), J2=J2, cdt=cdt, dnu=dnu)

    if bands is not None or not p.get("freq_step", True):  # no step 3 (nor its cap)
        return (J2, Hx2, Hy2, fx_out, fy_out), 0.0

    # step 3, a dense BDF1 solve per cell in the printed leakage form
    half = 0.5 * dnu  # delta nu_k on either side of a midpoint centre
    pmax = 0.0
    J3 = J2.copy()
    Hx3 = Hx2.copy()
    Hy3 = Hy2.copy()

    def phiL(P):
        return -math.expm1(-P)

    def phiR(P):
        return -math.expm1(P)

    def chiL(P):
        return 1.0 if P == 0.0 else phiL(P) / P

    def chiR(P):
        return -1.0 if P == 0.0 else phiR(P) / P

    for j in range(ny):
        for i in range(nx):
            if alpha[j, i] > 0.0:
                dD = dnuDc[j, i]
                K = 0.5 * dD * dD * alpha[j, i] * Hkc[:, j, i]
                Rk = HPL / (KB * Tc[j, i]) - 2.0 / nubar if p["recoil"] else np.zeros(nb)
                Cc = np.empty(nb)
                for k in range(nb):
                    fx, fy = cap(*prim(J2[k, j, i], Hx2[k, j, i], Hy2[k, j, i]))
                    Dxx, Dxy, Dyy, _ = closure(fx, fy)
                    DdU = Dxx * gxx[j, i] + Dyy * gyy[j, i] + Dxy * gsh[j, i]
                    Cc[k] = K[k] * Rk[k] + nubar[k] / C * DdU
                P = Cc * half / K
                pmax = max(pmax, float(np.abs(P).max()))
                M = np.zeros((nb, nb))
                for k in range(nb):
                    M[k, k] = 1.0 / cdt
                    if k + 1 < nb:  # interface k+1/2
                        den = chiL(P[k]) * half[k] / K[k] - chiR(P[k + 1]) * half[k + 1] / K[k + 1]
                        M[k, k + 1] -= (1.0 - phiR(P[k + 1])) / den / dnu[k]
                        M[k, k] += (1.0 - phiL(P[k])) / den / dnu[k]
                    if k > 0:  # interface k-1/2
                        den = chiL(P[k - 1]) * half[k - 1] / K[k - 1] - chiR(P[k]) * half[k] / K[k]
                        M[k, k - 1] -= (1.0 - phiL(P[k - 1])) / den / dnu[k]
                        M[k, k] += (1.0 - phiR(P[k])) / den / dnu[k]
                Jn = np.linalg.solve(M, J2[:, j, i] / cdt)
                ratio = np.where(J2[:, j, i] > 0.0, Jn / np.where(J2[:, j, i] > 0, J2[:, j, i], 1.0), 0.0)
                J3[:, j, i] = Jn
                Hx3[:, j, i] = ratio * Hx2[:, j, i]
                Hy3[:, j, i] = ratio * Hy2[:, j, i]
            for k in range(nb):  # causality: |H| <= J after the step
                jv, h1, h2 = J3[k, j, i], Hx3[k, j, i], Hy3[k, j, i]
                hn = math.hypot(h1, h2)
                if jv <= 0.0:
                    Hx3[k, j, i] = Hy3[k, j, i] = 0.0
                elif hn > jv:
                    Hx3[k, j, i] = h1 * jv / hn
                    Hy3[k, j, i] = h2 * jv / hn
    return (J3, Hx3, Hy3, fx_out, fy_out), pmax


def _problem(bc, seed):
    nx = ny = 8
    g = np.random.default_rng(seed)
    T = 1e4
    dnuD = line(T)[0]
    edges = np.linspace(-3.0, 3.0, 13) * dnuD  # 12 bins within 3 Doppler widths
    n_hi = 10.0 ** g.uniform(-1, 2, (ny, nx))  # |P| up to tens, where the printed form is finite
    p = dict(nx=nx, ny=ny, dx=1e16, edges=edges, T=T, n_hi=n_hi,
             rho_d=1e-24 * g.uniform(0, 1, (ny, nx)), p_d=10.0 ** g.uniform(-8, -4, (ny, nx)),
             ux=g.uniform(-50, 50, (ny, nx)) * 1e5, uy=g.uniform(-50, 50, (ny, nx)) * 1e5,
             lum=np.zeros((ny, nx)), kappa_abs=2.682e4, kappa_F=3.049e4, c_tilde=C, cfl=0.4,
             recoil=True, bc=bc)
    p["lum"][3:5, 3:5] = 1e38
    nb = edges.size - 1
    J = 1e-3 * np.exp(g.normal(0, 1.0, (nb, ny, nx)))
    th = g.uniform(0, 2 * np.pi, J.shape)
    f = g.uniform(0, 0.9, J.shape)
    return p, (J, J * f * np.cos(th), J * f * np.sin(th))


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1)])
def test_brute_force_substep_matches_oracle(bc):
    p, st = _problem(bc, 201 + sum(bc))
    O = oracle.Oracle(nx=p["nx"], ny=p["ny"], dx=p["dx"], edges=p["edges"], T=p["T"],
                      n_hi=p["n_hi"], rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"],
                      lum=p["lum"], kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"],
                      c_tilde=p["c_tilde"], cfl=p["cfl"], recoil=True, bc=bc)
    ref = O.substep(*st)[:5]
    got, pmax = brute_substep(p, *st)
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        scale = np.abs(b).max()
        assert scale > 0
        err = np.abs(a - b).max() / scale
        assert err < 1e-12, (n, err)
    # the problem reaches the upwind regime of the frequency step
    assert pmax > 5.0


def brute_substep_cyl(p, J, Hx, Hy, prune=0.0, diag=None):
    """The same substep on the axisymmetric grid (x = R from the axis, y = Z
    from the midplane, per-radian finite volumes): R faces of area R dZ, Z faces
    (R+^2 - R-^2)/2, volume (R+^2 - R-^2) dZ / 2, centroid distances in tau, the
    hoop source -K_phiphi <1/R> in the H_R balance and D_phiphi <u_R/R> in the
    work and Doppler terms; the axis and the midplane are mirrors.  prune: as
    for the Cartesian grid, the bin energies weighted by the ring volumes.
    diag: as for the Cartesian grid, with the geometry (R faces, volumes).
    p["temp"]: per-cell temperatures, every A0 table per cell."""
    nx, ny, dx = p["nx"], p["ny"], p["dx"]
    e = p["edges"]
    nb = e.size - 1
    dnu = np.diff(e)
    nubar = NU0 + 0.5 * (e[1:] + e[:-1])
    Tc = p.get("temp")
    Tc = np.full((ny, nx), p["T"]) if Tc is None else Tc
    Hk = np.empty((nb, ny, nx))
    w = np.empty((nb, ny, nx))
    dnuD = np.empty((ny, nx))
    s0 = np.empty((ny, nx))
    for j in range(ny):
        for i in range(nx):
            dD, av, sg = line(Tc[j, i])
            x = e / dD
            h = (I_voigt(x[1:], av) - I_voigt(x[:-1], av)) / (dnu / dD)
            ww = h * (dnu / dD)
            Hk[:, j, i] = h
            w[:, j, i] = ww / ww.sum()
            dnuD[j, i] = dD
            s0[j, i] = sg
    alpha = p["n_hi"] * s0
    rho, pd, ux, uy, lum = p["rho_d"], p["p_d"], p["ux"], p["uy"], p["lum"]
    kabs, kF = p["kappa_abs"], p["kappa_F"]
    ct = p["c_tilde"]
    umax = np.hypot(ux, uy).max()
    dt = (p["cfl"] / 2.0) * dx / (ct + umax)
    cdt = ct * dt
    bc = p["bc"]
    Rf = np.arange(nx + 1) * dx                      # R faces
    AZ = 0.5 * (Rf[1:] ** 2 - Rf[:-1] ** 2)          # Z-face areas
    Vol = AZ * dx
    Rbar = (2.0 / 3.0) * (Rf[1:] ** 3 - Rf[:-1] ** 3) / (Rf[1:] ** 2 - Rf[:-1] ** 2)

    def uR(i, j):  # with the axis mirror (u_R flips) and copied outer ghosts
        if i < 0:
            return -ux[min(max(j, -1 - j) if j < 0 else j, ny - 1), -1 - i]
        return ux[min(j if j >= 0 else -1 - j, ny - 1), min(i, nx - 1)]

    def uZ(i, j):  # with the midplane mirror (u_Z flips) and copied outer ghosts
        ii = min(i if i >= 0 else -1 - i, nx - 1)
        if j < 0:
            return -uy[-1 - j, ii]
        return uy[min(j, ny - 1), ii]

    gxx = np.zeros((ny, nx))
    gyy = np.zeros((ny, nx))
    gsh = np.zeros((ny, nx))
    gphi = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            gxx[j, i] = (uR(i + 1, j) - uR(i - 1, j)) / (2 * dx)
            gyy[j, i] = (uZ(i, j + 1) - uZ(i, j - 1)) / (2 * dx)
            gsh[j, i] = (uR(i, j + 1) - uR(i, j - 1)) / (2 * dx) + (uZ(i + 1, j) - uZ(i - 1, j)) / (2 * dx)
            fl = 0.5 * (uR(i - 1, j) + uR(i, j))
            fr = 0.5 * (uR(i, j) + uR(i + 1, j))
            gphi[j, i] = (fl + fr) / (Rf[i] + Rf[i + 1])

    J1 = np.empty_like(J)
    Hx1 = np.empty_like(J)
    Hy1 = np.empty_like(J)
    W = np.zeros((nb, ny, nx))
    FRJ = np.zeros((nb, ny, nx + 1))
    FZJ = np.zeros((nb, ny + 1, nx))
    Ek = dnu * (J * Vol[None, None, :]).sum(axis=(1, 2))
    on = Ek > prune * Ek.sum() if prune > 0.0 else np.ones(nb, bool)
    for k in range(nb):
        if not on[k]:  # a pruned bin keeps its state through step 1
            J1[k], Hx1[k], Hy1[k] = J[k], Hx[k], Hy[k]
            continue
        aF = alpha * Hk[k] + rho * kF

        def cell(i, j, axis):
            # (J, f_n, f_t), u_n, alpha_F of a (ghost) cell; axis 0: n = R, axis 1: n = Z
            flipR = i < 0
            flipZ = j < 0
            ii = -1 - i if i < 0 else min(i, nx - 1)
            jj = -1 - j if j < 0 else min(j, ny - 1)
            vac = (i >= nx and bc[1] == 1) or (j >= ny and bc[3] == 1)
            u = (-1.0 if flipR else 1.0) * ux[jj, ii] if axis == 0 else (-1.0 if flipZ else 1.0) * uy[jj, ii]
            if vac:
                return (0.0, 0.0, 0.0), u, aF[jj, ii]
            jv = J[k, jj, ii]
            hR = (-1.0 if flipR else 1.0) * Hx[k, jj, ii]
            hZ = (-1.0 if flipZ else 1.0) * Hy[k, jj, ii]
            fR, fZ = prim(jv, hR, hZ)
            return ((jv, fR, fZ) if axis == 0 else (jv, fZ, fR)), u, aF[jj, ii]

        def face(q, u0, u1, a0, a1, d0, d1):
            (Jm, nm, tm), (J0, n0, t0), (Jp, n1, t1), (J2, n2, t2) = q
            JL = J0 + 0.5 * minmod(J0 - Jm, Jp - J0)
            JR = Jp - 0.5 * minmod(Jp - J0, J2 - Jp)
            nL = n0 + 0.5 * minmod(n0 - nm, n1 - n0)
            tL = t0 + 0.5 * minmod(t0 - tm, t1 - t0)
            nR = n1 - 0.5 * minmod(n1 - n0, n2 - n1)
            tR = t1 - 0.5 * minmod(t1 - t0, t2 - t1)
            nL, tL = cap(nL, tL)
            nR, tR = cap(nR, tR)
            HnL, HtL, HnR, HtR = JL * nL, JL * tL, JR * nR, JR * tR
            DnnL, DntL, _, _ = closure(nL, tL)
            DnnR, DntR, _, _ = closure(nR, tR)
            tau = a0 * d0 + a1 * d1
            eps = (0.2 + tau) / (0.2 + tau + tau * tau)
            diff = (1.0 - eps) * (Jp - J0) / (3.0 * tau) if tau > 0.0 else 0.0
            wf = 0.5 * (u0 + u1) / C
            up = wf > 0.0
            FJ = eps * 0.5 * (HnL + HnR) - eps * 0.5 * (JR - JL) - diff + wf * (JL if up else JR)
            FN = 0.5 * (DnnL * JL + DnnR * JR) - eps * 0.5 * (HnR - HnL) + wf * (HnL if up else HnR)
            FT = 0.5 * (DntL * JL + DntR * JR) - eps * 0.5 * (HtR - HtL) + wf * (HtL if up else HtR)
            return FJ, FN, FT

        FR = np.zeros((3, ny, nx + 1))
        for j in range(ny):
            for i in range(nx + 1):  # R face i between cells i-1 and i
                cs = [cell(i - 2 + m, j, 0) for m in range(4)]
                left = -Rbar[0] if i == 0 else Rbar[i - 1]
                right = Rbar[nx - 1] + dx if i == nx else Rbar[i]
                FR[:, j, i] = face([c[0] for c in cs], cs[1][1], cs[2][1], cs[1][2], cs[2][2],
                                   Rf[i] - left, right - Rf[i])
        FZ = np.zeros((3, ny + 1, nx))
        for j in range(ny + 1):
            for i in range(nx):
                cs = [cell(i, j - 2 + m, 1) for m in range(4)]
                FZ[:, j, i] = face([c[0] for c in cs], cs[1][1], cs[2][1], cs[1][2], cs[2][2],
                                   dx / 2.0, dx / 2.0)
        FRJ[k], FZJ[k] = FR[0], FZ[0]
        for j in range(ny):
            for i in range(nx):
                jv = J[k, j, i]
                fx, fy = cap(*prim(jv, Hx[k, j, i], Hy[k, j, i]))
                Dxx, Dxy, Dyy, Dpp = closure(fx, fy)
                Wc = (Dxx * gxx[j, i] + Dyy * gyy[j, i] + Dxy * gsh[j, i] + Dpp * gphi[j, i]) * jv
                W[k, j, i] = Wc

                def div(fr, fz):
                    return ((Rf[i + 1] * dx * fr[j, i + 1] - Rf[i] * dx * fr[j, i])
                            + AZ[i] * (fz[j + 1, i] - fz[j, i])) / Vol[i]
                invR = dx * dx / Vol[i]
                J1[k, j, i] = jv - cdt * (div(FR[0], FZ[0]) + Wc / C)
                Hx1[k, j, i] = Hx[k, j, i] - cdt * (div(FR[1], FZ[2]) - Dpp * jv * invR)
                Hy1[k, j, i] = Hy[k, j, i] - cdt * div(FR[2], FZ[1])

    aH = alpha[None] * Hk
    kap = rho[None] * kabs + pd[None] * aH
    aFk = aH + rho[None] * kF
    js = (lum / (2.0 * math.pi * Vol[None, :]))[None] * w / (4.0 * math.pi * dnu[:, None, None])
    J2 = (J1 + cdt * js) / (1.0 + cdt * kap)
    Hx2 = Hx1 / (1.0 + cdt * aFk)
    Hy2 = Hy1 / (1.0 + cdt * aFk)
    fcoef = 4.0 * math.pi / (C * ct * dt)
    fx_out = fcoef * (dnu[:, None, None] * (Hx1 - Hx2)).sum(axis=0)
    fy_out = fcoef * (dnu[:, None, None] * (Hy1 - Hy2)).sum(axis=0)
    if diag is not None:
        shape = (nb, ny, nx)
        diag.update(FXJ=FRJ, FYJ=FZJ, W=W, kap=np.broadcast_to(kap, shape),
                    js=np.broadcast_to(js, shape), J2=J2, cdt=cdt, dnu=dnu, Rf=Rf, AZ=AZ,
                    Vol=Vol)
    if not p.get("freq_step", True):
        return (J2, Hx2, Hy2), fx_out, fy_out
    # step 3 with D_phiphi <u_R/R> in the Doppler term: the Cartesian routine's
    # solve, on gradients that include the hoop part
    q = dict(p, _grads=(gxx, gyy, gsh, gphi))
    return _freq_and_cap(q, J2, Hx2, Hy2, Hk, dnu, nubar, dnuD, alpha, cdt, Tc), fx_out, fy_out


def _freq_and_cap(p, J2, Hx2, Hy2, Hk, dnu, nubar, dnuD, alpha, cdt, T):
    # Hk [bin][cell], dnuD and T per cell
    nb = dnu.size
    ny, nx = alpha.shape
    gxx, gyy, gsh, gphi = p["_grads"]
    half = 0.5 * dnu
    J3, Hx3, Hy3 = J2.copy(), Hx2.copy(), Hy2.copy()

    def phiL(P):
        return -math.expm1(-P)

    def phiR(P):
        return -math.expm1(P)

    def chiL(P):
        return 1.0 if P == 0.0 else phiL(P) / P

    def chiR(P):
        return -1.0 if P == 0.0 else phiR(P) / P

    for j in range(ny):
        for i in range(nx):
            if alpha[j, i] > 0.0:
                K = 0.5 * dnuD[j, i] ** 2 * alpha[j, i] * Hk[:, j, i]
                hkT = HPL / (KB * T[j, i])
                Rk = hkT - 2.0 / nubar if p["recoil"] else np.zeros(nb)
                Cc = np.empty(nb)
                for k in range(nb):
                    fx, fy = cap(*prim(J2[k, j, i], Hx2[k, j, i], Hy2[k, j, i]))
                    Dxx, Dxy, Dyy, Dpp = closure(fx, fy)
                    DdU = Dxx * gxx[j, i] + Dyy * gyy[j, i] + Dxy * gsh[j, i] + Dpp * gphi[j, i]
                    Cc[k] = K[k] * Rk[k] + nubar[k] / C * DdU
                P = Cc * half / K
                M = np.zeros((nb, nb))
                for k in range(nb):
                    M[k, k] = 1.0 / cdt
                    if k + 1 < nb:
                        den = chiL(P[k]) * half[k] / K[k] - chiR(P[k + 1]) * half[k + 1] / K[k + 1]
                        M[k, k + 1] -= (1.0 - phiR(P[k + 1])) / den / dnu[k]
                        M[k, k] += (1.0 - phiL(P[k])) / den / dnu[k]
                    if k > 0:
                        den = chiL(P[k - 1]) * half[k - 1] / K[k - 1] - chiR(P[k]) * half[k] / K[k]
                        M[k, k - 1] -= (1.0 - phiL(P[k - 1])) / den / dnu[k]
                        M[k, k] += (1.0 - phiR(P[k])) / den / dnu[k]
                Jn = np.linalg.solve(M, J2[:, j, i] / cdt)
                Jo = J2[:, j, i]
                ratio = np.where(Jo > 0.0, Jn / np.where(Jo > 0, Jo, 1.0), 0.0)
                J3[:, j, i] = Jn
                Hx3[:, j, i] = ratio * Hx2[:, j, i]
                Hy3[:, j, i] = ratio * Hy2[:, j, i]
            for k in range(nb):
                jv, h1, h2 = J3[k, j, i], Hx3[k, j, i], Hy3[k, j, i]
                hn = math.hypot(h1, h2)
                if jv <= 0.0:
                    Hx3[k, j, i] = Hy3[k, j, i] = 0.0
                elif hn > jv:
                    Hx3[k, j, i] = h1 * jv / hn
                    Hy3[k, j, i] = h2 * jv / hn
    return J3, Hx3, Hy3


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 0, 1)])
def test_brute_force_axisymmetric_substep_matches_oracle(bc):
    p, st = _problem(bc, 211 + sum(bc))
    p["geometry"] = 1
    O = oracle.Oracle(nx=p["nx"], ny=p["ny"], dx=p["dx"], edges=p["edges"], T=p["T"],
                      n_hi=p["n_hi"], rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"],
                      lum=p["lum"], kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"],
                      c_tilde=p["c_tilde"], cfl=p["cfl"], recoil=True, bc=bc, geometry=1)
    ref = O.substep(*st)[:5]
    (J3, Hx3, Hy3), fx, fy = brute_substep_cyl(p, *st)
    for a, b, n in zip((J3, Hx3, Hy3, fx, fy), ref, ("J", "Hx", "Hy", "fx", "fy")):
        scale = np.abs(b).max()
        assert scale > 0
        err = np.abs(a - b).max() / scale
        assert err < 1e-12, (n, err)


def test_brute_force_temperature_field_matches_oracle():
    # per-cell temperatures from 5e3 K to 3e4 K (colder cells push the Peclet
    # numbers of this grid past the printed form's range): every A0 table per cell
    p, st = _problem((1, 0, 0, 1), 221)
    g = np.random.default_rng(222)
    p["temp"] = 10.0 ** g.uniform(np.log10(5e3), np.log10(3e4), (p["ny"], p["nx"]))
    O = oracle.Oracle(nx=p["nx"], ny=p["ny"], dx=p["dx"], edges=p["edges"], T=p["T"],
                      n_hi=p["n_hi"], rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"],
                      lum=p["lum"], kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"],
                      c_tilde=p["c_tilde"], cfl=p["cfl"], recoil=True, bc=p["bc"], temp=p["temp"])
    ref = O.substep(*st)[:5]
    got, pmax = brute_substep(p, *st)
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        scale = np.abs(b).max()
        err = np.abs(a - b).max() / scale
        assert err < 1e-12, (n, err)


def _per_bin_err(a, b):
    # worst error over the bin planes, each relative to its own largest value
    return max(np.abs(a[k] - b[k]).max() / np.abs(b[k]).max() for k in range(b.shape[0]))


CUT = 1e-10


@pytest.mark.parametrize("geometry", [0, 1])
def test_brute_force_pruning_matches_oracle(geometry):
    # Bins of unequal width (quadratic in nu), no sources, no step 3 (so that
    # each bin plane shows its own step 1).  Bins 0, 4, 11 hold ~1e-15 of the
    # energy; bin 6 (the narrowest) holds 0.4 cut and bin 8 holds 2.5 cut of
    # sum_k dnu_k sum_cells w J_k, w the ring volume on the axisymmetric grid,
    # where bin 6 lives on the axis column only.  Bin 6 is pruned and bin 8 is
    # not; leaving out dnu or w, or comparing with the mean bin, flips one of
    # the two decisions, and so does a reversed comparison.
    bc = (1, 0, 0, 1) if geometry == 0 else (0, 1, 0, 1)
    p, (J, Hx, Hy) = _problem(bc, 231 + geometry)
    dnuD = line(p["T"])[0]
    x = np.linspace(-1.0, 1.0, 13)
    p["edges"] = 3.0 * dnuD * np.sign(x) * x * x
    p["lum"] = np.zeros_like(p["lum"])
    p["freq_step"] = False
    nx, ny = p["nx"], p["ny"]
    dnu = np.diff(p["edges"])
    Vol = 0.5 * (2 * np.arange(nx) + 1) * p["dx"] ** 3 if geometry == 1 else np.ones(nx)
    for k in (0, 4, 11):
        J[k] *= 1e-14
        Hx[k] *= 1e-14
        Hy[k] *= 1e-14

    def energies(J, w_col, with_dnu=True):
        return (dnu if with_dnu else 1.0) * (J * w_col[None, None, :]).sum(axis=(1, 2))

    g = np.random.default_rng(233)
    J[6] = J[8] = 0.0
    Erest = energies(J, Vol).sum()
    for k, share in ((6, 0.4 * CUT), (8, 2.5 * CUT)):
        plane = np.zeros((ny, nx))
        if geometry == 1 and k == 6:
            plane[:, 0] = 1.0
        else:
            plane[:] = np.exp(g.normal(0, 0.3, (ny, nx)))
        S = (plane * Vol[None, :]).sum()
        J[k] = plane * (share * Erest / (1.0 - 2.9 * CUT)) / (dnu[k] * S)
        th = g.uniform(0, 2 * np.pi, (ny, nx))
        Hx[k] = 0.5 * J[k] * np.cos(th)
        Hy[k] = 0.5 * J[k] * np.sin(th)
    E = energies(J, Vol)
    assert E[6] / E.sum() == pytest.approx(0.4 * CUT, rel=1e-9)
    assert E[8] / E.sum() == pytest.approx(2.5 * CUT, rel=1e-9)
    # the readings that a plausible mistake takes all flip a decision
    Eu = energies(J, Vol, with_dnu=False)
    assert Eu[6] > 2.0 * CUT * Eu.sum()
    if geometry == 1:
        Ev = energies(J, np.ones(nx))
        assert Ev[6] > 2.0 * CUT * Ev.sum()
    assert E[6] > CUT * E.mean()
    st = (J, Hx, Hy)

    O = oracle.Oracle(nx=nx, ny=ny, dx=p["dx"], edges=p["edges"], T=p["T"], n_hi=p["n_hi"],
                      rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"], lum=p["lum"],
                      kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"], c_tilde=p["c_tilde"],
                      cfl=p["cfl"], recoil=True, freq_step=False, bc=bc, geometry=geometry,
                      prune=CUT)
    ref = O.substep(*st)[:5]
    if geometry == 0:
        got = brute_substep(p, *st, prune=CUT)[0]
        plain = brute_substep(p, *st)[0]
    else:
        (J3, Hx3, Hy3), fx, fy = brute_substep_cyl(p, *st, prune=CUT)
        got = (J3, Hx3, Hy3, fx, fy)
        (J3, Hx3, Hy3), fx, fy = brute_substep_cyl(p, *st)
        plain = (J3, Hx3, Hy3, fx, fy)
    for a, b, n in zip(got[:3], ref[:3], ("J", "Hx", "Hy")):
        err = _per_bin_err(a, b)
        assert err < 1e-12, (n, err)
    for a, b, n in zip(got[3:], ref[3:], ("fx", "fy")):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err < 1e-12, (n, err)
    # without pruning the skipped bins come out far from the oracle's
    for k in (0, 4, 6, 11):
        assert np.abs(plain[0][k] - ref[0][k]).max() > 1e-6 * np.abs(ref[0][k]).max(), k
    assert np.abs(plain[0][8] - ref[0][8]).max() < 1e-12 * np.abs(ref[0][8]).max()


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_brute_force_bands_match_oracle(bc):
    # three broad bands (Sec. 3): per-[band][cell] flux opacity with optical
    # depths 1e-2 to 1e2 per half cell, absorption 10-100 % of it, and an
    # emissivity that supplies a J of the state's order in one step
    nx = ny = 8
    dx = 1e16
    g = np.random.default_rng(241 + sum(bc))
    nb = 3
    aF = 10.0 ** g.uniform(-2, 2, (nb, ny, nx)) * 2.0 / dx
    kap = aF * g.uniform(0.1, 1.0, aF.shape)
    js = 5e-19 * g.uniform(0, 1, aF.shape)
    ux = g.uniform(-300, 300, (ny, nx)) * 1e5
    uy = g.uniform(-300, 300, (ny, nx)) * 1e5
    J = 1e-3 * np.exp(g.normal(0, 1.0, (nb, ny, nx)))
    th = g.uniform(0, 2 * np.pi, J.shape)
    f = g.uniform(0, 0.9, J.shape)
    st = (J, J * f * np.cos(th), J * f * np.sin(th))
    O = oracle.Oracle.for_bands(nx=nx, ny=ny, dx=dx, alpha_F=aF, kappa=kap, emissivity=js,
                                ux=ux, uy=uy, cfl=0.4, bc=bc)
    ref = O.substep(*st)[:5]
    z = np.zeros((ny, nx))
    p = dict(nx=nx, ny=ny, dx=dx, T=1e4, n_hi=z, rho_d=z, p_d=z, ux=ux, uy=uy, lum=z,
             kappa_abs=0.0, kappa_F=0.0, c_tilde=C, cfl=0.4, bc=bc)
    got = brute_substep(p, *st, bands=(aF, kap, js))[0]
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        err = _per_bin_err(a, b) if a.ndim == 3 else np.abs(a - b).max() / np.abs(b).max()
        assert err < 1e-12, (n, err)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 0, 0, 1)])
def test_brute_force_gray_group_matches_oracle(bc):
    # one gray group: the band equations with alpha_F = alpha eta + rho kappa_F,
    # kappa = rho kappa_abs + p_d alpha eta and j = L / (4 pi V), where
    # eta = sum_k w_k <H>_k over the bins of the grid (App. A tables)
    p, st = _problem(bc, 251 + sum(bc))
    e = p["edges"]
    dD, av, s0 = line(p["T"])
    xx = e / dD
    h = (I_voigt(xx[1:], av) - I_voigt(xx[:-1], av)) / (np.diff(e) / dD)
    w = h * np.diff(e) / dD
    w = w / w.sum()
    eta = float((w * h).sum())
    alpha = p["n_hi"] * s0
    aF = (alpha * eta + p["rho_d"] * p["kappa_F"])[None]
    kap = (p["rho_d"] * p["kappa_abs"] + p["p_d"] * alpha * eta)[None]
    js = (p["lum"] / (4.0 * math.pi * p["dx"] ** 3))[None]
    st1 = tuple(np.ascontiguousarray(a[5:6]) for a in st)
    O = oracle.Oracle(nx=p["nx"], ny=p["ny"], dx=p["dx"], edges=e, T=p["T"], n_hi=p["n_hi"],
                      rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"], lum=p["lum"],
                      kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"], c_tilde=p["c_tilde"],
                      cfl=p["cfl"], recoil=True, bc=bc, gray=True)
    assert O.nb == 1
    ref = O.substep(*st1)[:5]
    got = brute_substep(p, *st1, bands=(aF, kap, js))[0]
    for a, b, n in zip(got, ref, ("J", "Hx", "Hy", "fx", "fy")):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err < 1e-12, (n, err)


@pytest.mark.parametrize("bc", [(1, 0, 0, 1), (0, 1, 1, 0)])
def test_brute_force_bookkeeping_and_spectrum_match_oracle(bc):
    # The photon bookkeeping of one substep, in erg (4 pi V / c per unit of
    # sum_k dnu_k J_k): emission c_tilde dt j, absorption c_tilde dt kappa J'',
    # work c_tilde dt W / c, and the emergent spectrum, the J flux through each
    # outer face (x- rows, x+ rows, y- columns, y+ columns) per bin, whose sum
    # is the outflow; e_after from the state after step 3.
    p, st = _problem(bc, 261 + bc[0])
    O = oracle.Oracle(nx=p["nx"], ny=p["ny"], dx=p["dx"], edges=p["edges"], T=p["T"],
                      n_hi=p["n_hi"], rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"],
                      lum=p["lum"], kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"],
                      c_tilde=p["c_tilde"], cfl=p["cfl"], recoil=True, bc=bc)
    O.spectrum_on()
    out = O.substep(*st)
    d, spec = out[5], O.spectrum.copy()
    dg = {}
    (J3, Hx3, Hy3, fxb, fyb), _ = brute_substep(p, *st, diag=dg)
    nx, ny, dx = p["nx"], p["ny"], p["dx"]
    eunit = 4.0 * math.pi * dx ** 3 / C
    cdt, dnu = dg["cdt"], dg["dnu"]
    per_bin = eunit * cdt * dnu / dx
    faces = np.concatenate([-dg["FXJ"][:, :, 0], dg["FXJ"][:, :, nx],
                            -dg["FYJ"][:, 0, :], dg["FYJ"][:, ny, :]], axis=1) * per_bin[:, None]
    assert spec.shape == faces.shape == (dnu.size, 2 * (nx + ny))
    assert np.abs(spec - faces).max() <= 1e-12 * np.abs(faces).max()
    want = {
        "e_before": eunit * (dnu[:, None, None] * st[0]).sum(),
        "e_after": eunit * (dnu[:, None, None] * J3).sum(),
        "emitted": eunit * cdt * (dnu[:, None, None] * dg["js"]).sum(),
        "absorbed": eunit * cdt * (dnu[:, None, None] * dg["kap"] * dg["J2"]).sum(),
        "work": eunit * cdt * (dnu[:, None, None] * dg["W"]).sum() / C,
        "outflow": faces.sum(),
    }
    # the force integrals, |f| dV and f . r_hat dV with r from the box centre
    x = (np.arange(nx) + 0.5) * dx - 0.5 * nx * dx
    y = (np.arange(ny) + 0.5) * dx - 0.5 * ny * dx
    X, Y = np.meshgrid(x, y)
    want["force_abs"] = (np.hypot(fxb, fyb) * dx ** 3).sum()
    want["force_radial"] = ((fxb * X + fyb * Y) / np.hypot(X, Y) * dx ** 3).sum()
    for name, v in want.items():
        assert d[name] == pytest.approx(v, rel=1e-12), name
    # every source emits L dt c_tilde / c in total, whatever the geometry
    assert d["emitted"] == pytest.approx(p["lum"].sum() * cdt / C, rel=1e-12)
    # realisability after the causality cap of step 3
    hn = np.hypot(Hx3, Hy3)
    assert d["max_f"] == pytest.approx((hn[J3 > 0] / J3[J3 > 0]).max(), rel=1e-12)
    assert d["max_f"] <= 1.0 + 1e-15 and d["n_unrealisable"] == 0


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 0, 1)])
def test_brute_force_axisymmetric_bookkeeping_matches_oracle(bc):
    # the same on the axisymmetric grid: cell energies weighted by the ring
    # volume 2 pi Vol, and the emergent spectrum through the outer R faces
    # (area 2 pi R_out dZ) and the outer Z faces (area 2 pi (R+^2 - R-^2)/2)
    p, st = _problem(bc, 271 + bc[1])
    O = oracle.Oracle(nx=p["nx"], ny=p["ny"], dx=p["dx"], edges=p["edges"], T=p["T"],
                      n_hi=p["n_hi"], rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"],
                      lum=p["lum"], kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"],
                      c_tilde=p["c_tilde"], cfl=p["cfl"], recoil=True, bc=bc, geometry=1)
    O.spectrum_on()
    d = O.substep(*st)[5]
    spec = O.spectrum.copy()
    dg = {}
    (J3, Hx3, Hy3), fxb, fyb = brute_substep_cyl(p, *st, diag=dg)
    nx, ny, dx = p["nx"], p["ny"], p["dx"]
    eu = 4.0 * math.pi / C
    cdt, dnu = dg["cdt"], dg["dnu"]
    ring = 2.0 * math.pi * dg["Vol"][None, None, :]
    per_bin = eu * 2.0 * math.pi * cdt * dnu
    faces = np.concatenate([dg["FXJ"][:, :, nx] * (dg["Rf"][nx] * dx),
                            dg["FYJ"][:, ny, :] * dg["AZ"][None, :]], axis=1) * per_bin[:, None]
    assert spec.shape == faces.shape == (dnu.size, nx + ny)
    assert np.abs(spec - faces).max() <= 1e-12 * np.abs(faces).max()
    want = {
        "e_before": eu * (dnu[:, None, None] * st[0] * ring).sum(),
        "e_after": eu * (dnu[:, None, None] * J3 * ring).sum(),
        "emitted": eu * cdt * (dnu[:, None, None] * dg["js"] * ring).sum(),
        "absorbed": eu * cdt * (dnu[:, None, None] * dg["kap"] * dg["J2"] * ring).sum(),
        "work": eu * cdt * (dnu[:, None, None] * dg["W"] * ring).sum() / C,
        "outflow": faces.sum(),
    }
    # the force integrals over the rings, r_hat from the origin (R, Z) = (0, 0)
    R = (np.arange(nx) + 0.5) * dx
    Z = (np.arange(ny) + 0.5) * dx
    RR, ZZ = np.meshgrid(R, Z)
    want["force_abs"] = (np.hypot(fxb, fyb) * ring[0]).sum()
    want["force_radial"] = ((fxb * RR + fyb * ZZ) / np.hypot(RR, ZZ) * ring[0]).sum()
    for name, v in want.items():
        assert d[name] == pytest.approx(v, rel=1e-12), name
    # every source emits L dt c_tilde / c in total, whatever the geometry
    assert d["emitted"] == pytest.approx(p["lum"].sum() * cdt / C, rel=1e-12)
    hn = np.hypot(Hx3, Hy3)
    assert d["max_f"] == pytest.approx((hn[J3 > 0] / J3[J3 > 0]).max(), rel=1e-12)
    assert d["max_f"] <= 1.0 + 1e-15 and d["n_unrealisable"] == 0


def test_brute_force_axisymmetric_temperature_field_matches_oracle():
    # the axisymmetric substep under per-cell temperatures (5e3 K to 3e4 K):
    # every A0 table per cell, the emission per ring volume
    p, st = _problem((0, 1, 0, 1), 281)
    g = np.random.default_rng(282)
    p["temp"] = 10.0 ** g.uniform(np.log10(5e3), np.log10(3e4), (p["ny"], p["nx"]))
    O = oracle.Oracle(nx=p["nx"], ny=p["ny"], dx=p["dx"], edges=p["edges"], T=p["T"],
                      n_hi=p["n_hi"], rho_d=p["rho_d"], p_d=p["p_d"], ux=p["ux"], uy=p["uy"],
                      lum=p["lum"], kappa_abs=p["kappa_abs"], kappa_F=p["kappa_F"],
                      c_tilde=p["c_tilde"], cfl=p["cfl"], recoil=True, bc=p["bc"], geometry=1,
                      temp=p["temp"])
    ref = O.substep(*st)[:5]
    (J3, Hx3, Hy3), fx, fy = brute_substep_cyl(p, *st)
    for a, b, n in zip((J3, Hx3, Hy3, fx, fy), ref, ("J", "Hx", "Hy", "fx", "fy")):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err < 1e-12, (n, err)
