"""FP64 CPU oracle for the velocity-potential boundary-integral solve.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this module.  The product
path (the CUDA library and its binding) never calls it and shares no code with
it.

What it computes is the plain definition of the discrete method of Ambrose,
Camassa, Marzuola, McLaughlin, Robinson & Wilkening (arXiv 2108.01786):

  * matrix entries directly from Table 1 (K_kj = Im{zeta_j'/2 cot((zeta_j - zeta_k)/2)},
    G_kj = Re{...}), the diagonal limit K_jj(a,a) = Im{zeta''/(2 zeta')} (Sec. 3.2),
    the trapezoidal collocation K_kj,ml = K_kj(alpha_km, alpha_jl)/M_j and the
    block system eq. lin:sys with diagonal -1/2 I (surface), +1/2 I (solids) and
    the finite-rank correction -E_m on obstacle blocks (Sec. 3.3, eq. AB:cor);
  * the right-hand side of eq. Awb: b_0 = phi~, b_k = -psi_mv(zeta_k);
  * a dense LU solve (LAPACK gesv, the paper's GEPP reference solver, Sec. 7.4);
  * the normal velocity U from eqs. d:phi:mv, d:phi:j, d:phi:0 (Sec. 3.4) with
    omega' and the Hilbert transform taken spectrally (numpy FFT);
  * psi|_k = <1_k, omega> (eq. psi:k), the energy of eq. E:formula (Sec. 5.2),
    and the Cauchy-integral / Helsing-Ojala evaluation of Phi' at targets
    (Sec. 5.1, eq. helsing:quad; App. F).

The cotangent is evaluated directly, 0.5/tan(z/2), on the FP64 difference of the
two nodes; no separable or exponential rewriting is used here.

Readings where the paper is silent:
  * Nyquist mode (even M): the derivative and Hilbert symbols are set to 0 at
    k = M/2.
  * The diagonal of G_00 in eq. d:phi:0 is the limit Re{zeta''/(2 zeta')}.
  * psi on the free surface (needed by the energy) is Im Phi~(zeta_0^-) + psi_mv,
    with Im Phi~(zeta_0^-) = 1/2 H omega_0 - G_00 omega_0 + sum_{j>=1} K_0j omega_j,
    obtained from Table 1 rows 1-2 and the Plemelj step of eq. plemelj:ver2.
"""
from __future__ import annotations

import numpy as np
from types import SimpleNamespace

TWO_PI = 2.0 * np.pi


# ---------------------------------------------------------------------------
# helpers on the concatenated node arrays
# ---------------------------------------------------------------------------

def offsets(M):
    return np.concatenate([[0], np.cumsum(M)]).astype(np.int64)


def block_ids(M):
    return np.concatenate([np.full(m, k, dtype=np.int64) for k, m in enumerate(M)])


def half_cot(z):
    """(1/2) cot(z/2): the periodic Cauchy kernel, Mittag-Leffler sum over images
    (Sec. 3, the PV sum of 1/(zeta + 2 pi k - z))."""
    return 0.5 / np.tan(0.5 * z)


# ---------------------------------------------------------------------------
# matrix of eq. lin:sys
# ---------------------------------------------------------------------------

def kernel_rows(geom, rows):
    """Rows `rows` of the discrete operator A (eq. lin:sys), as a dense array.

    A = diag(-1/2 on block 0, +1/2 on blocks >= 1)
        + [K_00 | G_0j ; -G_k0 | K_kj]  (entries of Table 1 / M_j)
        - E_k on obstacle diagonal blocks (k >= 2), E_k = e e^T / M_k.
    """
    M = list(geom.M)
    bid = block_ids(M)
    N = len(bid)
    rows = np.asarray(rows, dtype=np.int64)
    zt = geom.zeta[rows][:, None]            # zeta_k(alpha_km)  (target)
    zs = geom.zeta[None, :]                  # zeta_j(alpha_jl)  (source)
    dzs = geom.dzeta[None, :]
    kr = bid[rows][:, None]
    js = bid[None, :]
    Mj = np.asarray(M, dtype=np.float64)[bid][None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        F = dzs * half_cot(zs - zt)          # zeta_j'(beta)/2 cot((zeta_j(beta)-zeta_k(alpha))/2)
    Kv, Gv = F.imag, F.real
    # block signs: K on (0,0) and (k>=1, j>=1); G_0j on (0, j>=1); -G_k0 on (k>=1, 0)
    A = np.where((kr == 0) & (js == 0), Kv,
        np.where(kr == 0, Gv,
        np.where(js == 0, -Gv, Kv)))
    # diagonal limit K_jj(alpha, alpha) = Im{zeta''/(2 zeta')}
    diag_cols = rows
    dlim = (geom.d2zeta[diag_cols] / (2.0 * geom.dzeta[diag_cols])).imag
    A[np.arange(len(rows)), diag_cols] = dlim
    A = A / Mj
    # +-1/2 I
    s = np.where(bid[rows] == 0, -0.5, 0.5)
    A[np.arange(len(rows)), diag_cols] += s
    # -E_k on obstacle diagonal blocks
    for i, r in enumerate(rows):
        k = bid[r]
        if k >= 2:
            A[i, bid == k] -= 1.0 / M[k]
    return A


def assemble(geom, chunk=1024):
    """Dense FP64 matrix of eq. lin:sys (N x N)."""
    N = geom.N
    A = np.empty((N, N), dtype=np.float64)
    for r0 in range(0, N, chunk):
        rows = np.arange(r0, min(N, r0 + chunk))
        A[rows] = kernel_rows(geom, rows)
    return A


# ---------------------------------------------------------------------------
# right-hand side of eq. Awb
# ---------------------------------------------------------------------------

def psi_cyl(z):
    """Im Phi_cyl(z) = -ln|1 - e^{iz}| (Sec. 3.1)."""
    return -np.log(np.abs(1.0 - np.exp(1j * z)))


def psi_mv(geom, flow, z):
    """Im Phi_mv(z) = V1 Im z + sum_j a_j psi_cyl(z - z_j) (eq. Phi:mv)."""
    out = flow.V1 * np.imag(z)
    for aj, zj in zip(flow.a, geom.zc):
        out = out + aj * psi_cyl(z - zj)
    return out


def rhs(geom, flow, phitilde):
    """b_0 = phi~ on the surface, b_k = -psi_mv(zeta_k) on solid boundaries (eq. Awb)."""
    M = list(geom.M)
    o = offsets(M)
    b = np.empty(geom.N, dtype=np.float64)
    b[: M[0]] = phitilde
    zsol = geom.zeta[M[0]:]
    b[M[0]:] = -psi_mv(geom, flow, zsol)
    return b


# ---------------------------------------------------------------------------
# spectral operators on one boundary (periodic, M points)
# ---------------------------------------------------------------------------

def wavenumbers(M):
    k = np.fft.fftfreq(M, d=1.0 / M)
    if M % 2 == 0:
        k[M // 2] = 0.0          # Nyquist mode dropped (reading: even M)
    return k


def d_alpha(f):
    """Spectral derivative of a 2pi-periodic sample vector."""
    k = wavenumbers(len(f))
    return np.real(np.fft.ifft(1j * k * np.fft.fft(f)))


def hilbert(f):
    """H f with symbol -i sgn(k) (Sec. 3.4)."""
    k = wavenumbers(len(f))
    return np.real(np.fft.ifft(-1j * np.sign(k) * np.fft.fft(f)))


def split(v, M):
    o = offsets(M)
    return [v[o[k]:o[k + 1]] for k in range(len(M))]


# ---------------------------------------------------------------------------
# solve and normal velocity
# ---------------------------------------------------------------------------

def solve_dense(A, b):
    """GEPP (LAPACK gesv)."""
    return np.linalg.solve(A, b)


def psi_k(geom, omega):
    """psi|_k = <1_k, omega> = (1/M_k) sum_l omega_k,l for obstacles k >= 2 (eq. psi:k)."""
    w = split(omega, geom.M)
    return np.array([w[k].mean() for k in range(2, len(geom.M))])


def normal_velocity(geom, flow, omega, targets=None):
    """U on the free surface: the sum of eqs. d:phi:mv, d:phi:j (j >= 1) and d:phi:0,
    divided by s_alpha = |zeta_0'|.  `targets` optionally restricts the output to
    a subset of surface node indices (each U_m is computed independently)."""
    M = list(geom.M)
    z0a, dz0a, d2z0a = geom.block(0)
    idx = np.arange(M[0]) if targets is None else np.asarray(targets, dtype=np.int64)
    z0, dz0, d2z0 = z0a[idx], dz0a[idx], d2z0a[idx]
    s_alpha = np.abs(dz0)
    w = split(omega, M)
    wp = [d_alpha(wk) for wk in w]                 # omega_j'
    # multi-valued part, eq. d:phi:mv
    term_mv = -(flow.V1 + 0.5 * np.sum(flow.a)) * dz0.imag
    for aj, zj in zip(flow.a, geom.zc):
        term_mv = term_mv + aj * np.real(half_cot(z0 - zj) * dz0)
    # j >= 1, eq. d:phi:j: (1/M_j) sum_l K_j0(beta_l, alpha) omega_j'(beta_l),
    # K_j0(beta, alpha) = Im{zeta_0'(alpha)/2 cot((zeta_0(alpha) - zeta_j(beta))/2)}
    term_j = np.zeros(len(idx))
    o = offsets(M)
    for j in range(1, len(M)):
        zj = geom.zeta[o[j]:o[j + 1]]
        Kj0 = np.imag(dz0[:, None] * half_cot(z0[:, None] - zj[None, :]))
        term_j += Kj0 @ wp[j] / M[j]
    # j = 0, eq. d:phi:0: -1/2 H omega_0' - (1/M_0) sum_l G_00(beta_l, alpha) omega_0'(beta_l)
    # G_00(beta, alpha) = Re{zeta_0'(alpha)/2 cot((zeta_0(alpha)-zeta_0(beta))/2) - 1/2 cot((alpha-beta)/2)}
    a0 = TWO_PI * np.arange(M[0]) / M[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.real(dz0[:, None] * half_cot(z0[:, None] - z0a[None, :])
                    - half_cot(a0[idx][:, None] - a0[None, :]))
    G[np.arange(len(idx)), idx] = np.real(d2z0 / (2.0 * dz0))
    term_0 = -0.5 * hilbert(wp[0])[idx] - G @ wp[0] / M[0]
    return (term_mv + term_j + term_0) / s_alpha


def solve(geom, flow, phitilde):
    """Full oracle solve: (omega, U, psi_k)."""
    A = assemble(geom)
    b = rhs(geom, flow, phitilde)
    omega = solve_dense(A, b)
    return omega, normal_velocity(geom, flow, omega), psi_k(geom, omega)


# ---------------------------------------------------------------------------
# stream function on the surface and the energy (Sec. 5.2)
# ---------------------------------------------------------------------------

def psi_surface(geom, flow, omega):
    """psi on Gamma_0 (from the fluid side): Im Phi~(zeta_0^-) + psi_mv(zeta_0)."""
    M = list(geom.M)
    o = offsets(M)
    z0, dz0, d2z0 = geom.block(0)
    w = split(omega, M)
    a0 = TWO_PI * np.arange(M[0]) / M[0]
    # G_00(alpha, beta) = Re{zeta_0'(beta)/2 cot((zeta_0(beta)-zeta_0(alpha))/2) - 1/2 cot((beta-alpha)/2)}
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.real(dz0[None, :] * half_cot(z0[None, :] - z0[:, None])
                    - half_cot(a0[None, :] - a0[:, None]))
    G[np.arange(M[0]), np.arange(M[0])] = np.real(d2z0 / (2.0 * dz0))
    out = 0.5 * hilbert(w[0]) - G @ w[0] / M[0]
    for j in range(1, len(M)):
        zj = geom.zeta[o[j]:o[j + 1]]
        dzj = geom.dzeta[o[j]:o[j + 1]]
        K0j = np.imag(dzj[None, :] * half_cot(zj[None, :] - z0[:, None]))
        out += K0j @ w[j] / M[j]
    return out + psi_mv(geom, flow, z0)


def phi_alpha_surface(geom, flow, phitilde):
    """d/dalpha of phi = phi~ + phi_mv along the surface; phi_mv' = Re{Phi_mv'(zeta) zeta'}
    with Phi_mv' = V1 + sum a_j (1/2 - i/2 cot((z - z_j)/2)) (eq. d:phi:cyl)."""
    z0, dz0, _ = geom.block(0)
    dPhi = flow.V1 + 0 * z0
    for aj, zj in zip(flow.a, geom.zc):
        dPhi = dPhi + aj * (0.5 - 1j * half_cot(z0 - zj))
    return d_alpha(phitilde) + np.real(dPhi * dz0)


def energy(geom, flow, phitilde, omega, tau=0.1, g=1.0, rho=1.0):
    """E of eq. E:formula by the trapezoidal rule on the M_0 surface points."""
    z0, dz0, _ = geom.block(0)
    s_alpha = np.abs(dz0)
    eta, xi_a = z0.imag, dz0.real
    psi0 = psi_surface(geom, flow, omega)
    phia = phi_alpha_surface(geom, flow, phitilde)
    integrand = rho * tau * s_alpha + 0.5 * rho * g * eta ** 2 * xi_a + 0.5 * psi0 * phia
    E = integrand.mean()
    E += 0.5 * np.sum(flow.a * psi_k(geom, omega))
    return E


# ---------------------------------------------------------------------------
# velocity at targets (Sec. 5.1): far-field Cauchy sums and Helsing-Ojala
# ---------------------------------------------------------------------------

def gammas(geom, omega):
    """gamma_0 = -omega_0', gamma_j = omega_j' (eq. gam:def)."""
    w = split(omega, geom.M)
    return [-d_alpha(w[0])] + [d_alpha(wk) for wk in w[1:]]


def dPhi_mv(geom, flow, z):
    """Phi_mv'(z) = V1 + sum_j a_j (1/2 - i/2 cot((z - z_j)/2))."""
    out = flow.V1 + 0 * np.asarray(z, dtype=np.complex128)
    for aj, zj in zip(flow.a, geom.zc):
        out = out + aj * (0.5 - 1j * half_cot(z - zj))   # eq. d:phi:cyl
    return out


def velocity_far(geom, flow, omega, z):
    """u - i v = Phi'(z) at interior targets by the plain trapezoidal sums of
    eqs. Phi:j:prime (j >= 1) and Phi:0:prime, plus Phi_mv'."""
    M = list(geom.M)
    o = offsets(M)
    w = split(omega, M)
    z = np.asarray(z, dtype=np.complex128)
    out = dPhi_mv(geom, flow, z)
    for j in range(len(M)):
        zj = geom.zeta[o[j]:o[j + 1]]
        wpj = d_alpha(w[j])
        S = half_cot(zj[None, :] - z[:, None]) @ wpj / M[j]
        out = out + (S / 1j if j == 0 else S)
    return out


def boundary_dphi(geom, flow, omega):
    """Boundary values Phi'(zeta_k(alpha_m)) = (phi_s - i phi_n) s_alpha / zeta_k'
    (eq. phi:prime) with s_alpha phi_s, s_alpha phi_n from eqs. dphij:dsk, dphij:dnk.

    In the velocity-potential formulation the gammas are obtained from omega
    first (eq. gam:def).  On the free surface the fluid is on the '-' side, so
    the jump terms use the lower sign; on solid boundaries phi_n = 0 is not
    imposed here but computed (it vanishes to the discretisation error).
    """
    M = list(geom.M)
    o = offsets(M)
    nb = len(M)
    gam = gammas(geom, omega)
    out = []
    for k in range(nb):
        zk = geom.zeta[o[k]:o[k + 1]]
        dzk = geom.dzeta[o[k]:o[k + 1]]
        d2zk = geom.d2zeta[o[k]:o[k + 1]]
        ak = TWO_PI * np.arange(M[k]) / M[k]
        # multi-valued part: s phi_mv,n and s phi_mv,s
        dPm = dPhi_mv(geom, flow, zk)
        sn = np.real(dPm * 1j * dzk)
        ss = np.real(dPm * dzk)
        for j in range(nb):
            zj = geom.zeta[o[j]:o[j + 1]]
            dzj = geom.dzeta[o[j]:o[j + 1]]
            aj = TWO_PI * np.arange(M[j]) / M[j]
            # C(beta, alpha) = zeta_k'(alpha)/2 cot((zeta_k(alpha) - zeta_j(beta))/2)
            with np.errstate(divide="ignore", invalid="ignore"):
                C = dzk[:, None] * half_cot(zk[:, None] - zj[None, :])
                if j == k:
                    C = C - half_cot(ak[:, None] - aj[None, :])   # Hilbert-regularised
                    C[np.arange(M[k]), np.arange(M[k])] = d2zk / (2.0 * dzk)
            Kjk = np.imag(C)   # K_jk(beta, alpha) (minus a real PV term when j == k)
            Gjk = np.real(C)   # G_jk(beta, alpha)
            g = gam[j]
            if j == 0:
                # eq. dphij:dnk (j=0 line) and dphij:dsk (j=0 line), '-' side on Gamma_0
                sn = sn + Gjk @ g / M[j]
                ss = ss + Kjk @ g / M[j]
                if k == 0:
                    sn = sn + 0.5 * hilbert(g)
                    ss = ss + 0.5 * g        # -/+ delta/2 gamma_0 with the lower sign
            else:
                sn = sn + Kjk @ g / M[j]
                ss = ss - Gjk @ g / M[j]
                if k == j:
                    sn = sn - 0.5 * g
                    ss = ss - 0.5 * hilbert(g)
        s = np.abs(dzk)
        out.append((ss / s - 1j * sn / s) * s / dzk)
    return out


def helsing_eval(geom, fvals, z):
    """Helsing-Ojala periodic quadrature, eq. helsing:quad.

    fvals: list of boundary values f(zeta_k(alpha_m)) per boundary.  The boundary
    of Omega must be positively oriented with respect to Omega: the free surface
    (fluid on its right) enters with -zeta_0', the bottom and the clockwise
    obstacles with +zeta_k' (reading of eq. res:thm; App. F).
    If z coincides with a node the node value is returned.
    """
    M = list(geom.M)
    o = offsets(M)
    z = np.asarray(z, dtype=np.complex128)
    num = np.zeros(z.shape, dtype=np.complex128)
    den = np.zeros(z.shape, dtype=np.complex128)
    hit = np.full(z.shape, -1, dtype=np.int64)
    for k in range(len(M)):
        zk = geom.zeta[o[k]:o[k + 1]]
        dzk = geom.dzeta[o[k]:o[k + 1]] * (-1.0 if k == 0 else 1.0)
        diff = zk[None, :] - z[:, None]
        exact = diff == 0
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = half_cot(diff) * dzk[None, :] / M[k]
        lam[exact] = 0.0
        num += lam @ fvals[k]
        den += lam.sum(axis=1)
        if exact.any():
            r, c = np.nonzero(exact)
            hit[r] = o[k] + c
    out = num / den
    allf = np.concatenate(fvals)
    out[hit >= 0] = allf[hit[hit >= 0]]
    return out


def cauchy_sum(geom, fvals, z):
    """(1/2 pi i) sum_k sigma_k sum_m (2 pi/M_k) f(zeta_km) 1/2 cot((zeta_km - z)/2) zeta_k'
    with sigma_0 = -1, sigma_k = +1: the trapezoidal Cauchy integral over the
    positively oriented boundary (eq. res:thm)."""
    M = list(geom.M)
    o = offsets(M)
    z = np.asarray(z, dtype=np.complex128)
    acc = np.zeros(z.shape, dtype=np.complex128)
    for k in range(len(M)):
        zk = geom.zeta[o[k]:o[k + 1]]
        dzk = geom.dzeta[o[k]:o[k + 1]] * (-1.0 if k == 0 else 1.0)
        acc += (half_cot(zk[None, :] - z[:, None]) * dzk[None, :]) @ fvals[k] * (TWO_PI / M[k])
    return acc / (2j * np.pi)


# ---------------------------------------------------------------------------
# vortex-sheet cross-check (Sec. 4.1): eq. lin:sys2 and eq. U:from:gam:j
# ---------------------------------------------------------------------------

def vs_normal_velocity(geom, flow, gamma0):
    """Given gamma_0, solve eq. lin:sys2 for gamma_1..gamma_N and return U from
    eq. U:from:gam:j.  Independent of the VP matrix: it uses the transposed
    kernels K_jk(beta, alpha), G_jk(beta, alpha) with weights 1/M_j (eq. KG:tmat)."""
    return vs_solve(geom, flow, gamma0)[0]


def vs_kernel_block(geom, j, k):
    """C[m, l] = zeta_k'(alpha_m)/2 cot((zeta_k(alpha_m) - zeta_j(beta_l))/2), the
    transposed kernel with the target on boundary k; for j == k the real part
    is regularised by 1/2 cot((alpha_m - beta_l)/2) and the diagonal is the
    limit zeta''/(2 zeta')."""
    M = list(geom.M)
    o = offsets(M)
    zk = geom.zeta[o[k]:o[k + 1]]
    dzk = geom.dzeta[o[k]:o[k + 1]]
    zj = geom.zeta[o[j]:o[j + 1]]
    with np.errstate(divide="ignore", invalid="ignore"):
        c = dzk[:, None] * half_cot(zk[:, None] - zj[None, :])
    if j == k:
        ak = TWO_PI * np.arange(M[k]) / M[k]
        with np.errstate(divide="ignore", invalid="ignore"):
            c = c - half_cot(ak[:, None] - ak[None, :])
        d2zk = geom.d2zeta[o[k]:o[k + 1]]
        c[np.arange(M[k]), np.arange(M[k])] = d2zk / (2.0 * dzk)
    return c


def vs_solve(geom, flow, gamma0):
    """(U, [gamma_1, ..., gamma_N]): eq. lin:sys2 and eq. U:from:gam:j."""
    M = list(geom.M)
    o = offsets(M)
    nb = len(M)

    def C(j, k):
        # C[m, l] = zeta_k'(alpha_m)/2 cot((zeta_k(alpha_m) - zeta_j(beta_l))/2)  (target on k)
        zk = geom.zeta[o[k]:o[k + 1]]
        dzk = geom.dzeta[o[k]:o[k + 1]]
        zj = geom.zeta[o[j]:o[j + 1]]
        with np.errstate(divide="ignore", invalid="ignore"):
            c = dzk[:, None] * half_cot(zk[:, None] - zj[None, :])
        if j == k:
            ak = TWO_PI * np.arange(M[k]) / M[k]
            with np.errstate(divide="ignore", invalid="ignore"):
                c = c - half_cot(ak[:, None] - ak[None, :])
            d2zk = geom.d2zeta[o[k]:o[k + 1]]
            c[np.arange(M[k]), np.arange(M[k])] = d2zk / (2.0 * dzk)
        return c

    def s_dphimv_dn(k):
        zk = geom.zeta[o[k]:o[k + 1]]
        dzk = geom.dzeta[o[k]:o[k + 1]]
        out = -(flow.V1 + 0.5 * np.sum(flow.a)) * dzk.imag
        for aj, zj in zip(flow.a, geom.zc):
            out = out + aj * np.real(half_cot(zk - zj) * dzk)
        return out

    ns = sum(M[1:])
    E = np.zeros((ns, ns))
    rhs_v = np.zeros(ns)
    os_ = offsets(M[1:])
    for kk, k in enumerate(range(1, nb)):
        rk = slice(os_[kk], os_[kk + 1])
        # -G_0k^* gamma_0 - s phi_mv,n
        rhs_v[rk] = -(np.real(C(0, k)) @ gamma0) / M[0] - s_dphimv_dn(k)
        for jj, j in enumerate(range(1, nb)):
            cj = slice(os_[jj], os_[jj + 1])
            E[rk, cj] = np.imag(C(j, k)) / M[j]
            if j == k:
                E[rk, cj] += -0.5 * np.eye(M[k])
    gam = np.linalg.solve(E, rhs_v)
    gam = split(gam, M[1:])
    c00 = C(0, 0)
    z0, dz0, _ = geom.block(0)
    tot = 0.5 * hilbert(gamma0) + np.real(c00) @ gamma0 / M[0] + s_dphimv_dn(0)
    for j in range(1, nb):
        tot = tot + np.imag(C(j, 0)) @ gam[j - 1] / M[j]
    return tot / np.abs(dz0), gam


# ---------------------------------------------------------------------------
# forward-mode directional derivatives of J = int U^2 d alpha (adjoint checks)
# ---------------------------------------------------------------------------

def d_half_cot(z):
    """d/dz [1/2 cot(z/2)] = -1/4 csc^2(z/2)."""
    s = np.sin(0.5 * z)
    return -0.25 / (s * s)


def objective(geom, flow, phitilde):
    """J = int_0^{2pi} U^2 d alpha by the trapezoidal rule on the surface nodes."""
    om, U, _ = solve(geom, flow, phitilde)
    return TWO_PI / geom.M[0] * np.sum(U * U), om, U


def directional_U(geom, flow, phitilde, dz, ddz, dd2z, dzc, dphit):
    """Forward-mode derivative of U along a direction of the inputs: dz, ddz,
    dd2z (complex, per node) are the changes of zeta, zeta', zeta''; dzc
    (complex, per obstacle) of the centres z_j in Phi_mv; dphit of phi~.
    Returns (U, dU)."""
    U, dUs = directional_U_many(geom, flow, phitilde, [(dz, ddz, dd2z, dzc, dphit)])
    return U, dUs[0]


def directional_U_many(geom, flow, phitilde, directions):
    """Forward-mode derivatives of U along several directions (tuples as in
    directional_U), sharing one GEPP factorisation of A.
    Every factor of the chain is differentiated by hand from its definition:
      A omega = b (eq. lin:sys, Table 1)  ->  d omega = A^{-1}(db - dA omega),
      U from eqs. d:phi:mv, d:phi:j, d:phi:0  ->  dU.
    The kernel derivative is d[1/2 cot(x/2)] = -1/4 csc^2(x/2).
    Returns (U, [dU, ...])."""
    import scipy.linalg as sla
    M = list(geom.M)
    N = geom.N
    bid = block_ids(M)
    o = offsets(M)
    A = assemble(geom)
    b = rhs(geom, flow, phitilde)
    lu = sla.lu_factor(A)
    om = sla.lu_solve(lu, b)
    U = normal_velocity(geom, flow, om)
    # direction-independent factors, formed once: 1/2 cot and its derivative
    # at every node difference (matrix), at surface-minus-source differences
    # (U sums) and the real cotangent of the G_00 regularisation
    zt, zs = geom.zeta[:, None], geom.zeta[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        Gm = half_cot(zs - zt)
        Gpm = d_half_cot(zs - zt)
    kr, js = bid[:, None], bid[None, :]
    z0, dz0, d2z0 = geom.block(0)
    s_alpha = np.abs(dz0)
    w = split(om, M)
    wp = [d_alpha(x) for x in w]
    a_sum = np.sum(flow.a)
    Cs, Cps = [None], [None]
    for j in range(1, len(M)):
        zj = geom.zeta[o[j]:o[j + 1]]
        Cs.append(half_cot(z0[:, None] - zj[None, :]))
        Cps.append(d_half_cot(z0[:, None] - zj[None, :]))
    a0 = TWO_PI * np.arange(M[0]) / M[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        C00 = half_cot(z0[:, None] - z0[None, :])
        Cp00 = d_half_cot(z0[:, None] - z0[None, :])
        G = np.real(dz0[:, None] * C00 - half_cot(a0[:, None] - a0[None, :]))
    ii = np.arange(M[0])
    G[ii, ii] = np.real(d2z0 / (2.0 * dz0))
    out = []
    for dz, ddz, dd2z, dzc, dphit in directions:
        # dA (off-diagonal kernel part and diagonal limit), weights 1/M_j
        dzt, dzs = dz[:, None], dz[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            dG = Gpm * (dzs - dzt)
            dF = ddz[None, :] * Gm + geom.dzeta[None, :] * dG
        dA = np.where((kr == 0) & (js == 0), dF.imag,
             np.where(kr == 0, dF.real, np.where(js == 0, -dF.real, dF.imag)))
        d1, d2 = geom.dzeta, geom.d2zeta
        ddiag = (dd2z / (2.0 * d1) - d2 * ddz / (2.0 * d1 * d1)).imag
        dA[np.arange(N), np.arange(N)] = ddiag
        dA = dA / np.asarray(M, float)[bid][None, :]
        # db: surface phi~, solids -psi_mv(zeta) with psi_mv = Im Phi_mv
        db = np.zeros(N)
        db[: M[0]] = dphit
        zsol = geom.zeta[M[0]:]
        dpsi = np.imag(flow.V1 * dz[M[0]:])
        for aj, zj, dzj in zip(flow.a, geom.zc, dzc):
            dc = 0.5 - 1j * half_cot(zsol - zj)          # Phi_cyl'(z - z_j)
            dpsi = dpsi + aj * np.imag(dc * (dz[M[0]:] - dzj))
        db[M[0]:] = -dpsi
        dom = sla.lu_solve(lu, db - dA @ om)
        # dU
        dz0_, ddz0, dd2z0 = dz[: M[0]], ddz[: M[0]], dd2z[: M[0]]
        ds = np.real(np.conj(dz0 / s_alpha) * ddz0)
        dw = split(dom, M)
        dwp = [d_alpha(x) for x in dw]
        dmv = -(flow.V1 + 0.5 * a_sum) * ddz0.imag
        mv = -(flow.V1 + 0.5 * a_sum) * dz0.imag
        for aj, zj, dzj in zip(flow.a, geom.zc, dzc):
            hc = half_cot(z0 - zj)
            mv = mv + aj * np.real(hc * dz0)
            dmv = dmv + aj * np.real(d_half_cot(z0 - zj) * (dz0_ - dzj) * dz0 + hc * ddz0)
        Nn = mv.copy()
        dN = dmv.copy()
        for j in range(1, len(M)):
            dzj = dz[o[j]:o[j + 1]]
            C = Cs[j]
            dC = Cps[j] * (dz0_[:, None] - dzj[None, :])
            K = np.imag(dz0[:, None] * C)
            dK = np.imag(ddz0[:, None] * C + dz0[:, None] * dC)
            Nn += K @ wp[j] / M[j]
            dN += (dK @ wp[j] + K @ dwp[j]) / M[j]
        with np.errstate(divide="ignore", invalid="ignore"):
            dC = Cp00 * (dz0_[:, None] - dz0_[None, :])
            dGm = np.real(ddz0[:, None] * C00 + dz0[:, None] * dC)
        dGm[ii, ii] = np.real(dd2z0 / (2.0 * dz0) - d2z0 * ddz0 / (2.0 * dz0 * dz0))
        Nn += -0.5 * hilbert(wp[0]) - G @ wp[0] / M[0]
        dN += -0.5 * hilbert(dwp[0]) - (dGm @ wp[0] + G @ dwp[0]) / M[0]
        out.append(dN / s_alpha - Nn * ds / s_alpha ** 2)
    return U, out


def directional_objective(geom, flow, phitilde, dz, ddz, dd2z, dzc, dphit):
    """dJ for J = (2 pi/M_0) sum U^2 along a direction: (4 pi/M_0) sum U dU."""
    U, dU = directional_U(geom, flow, phitilde, dz, ddz, dd2z, dzc, dphit)
    return 2.0 * TWO_PI / geom.M[0] * np.sum(U * dU)


# ---------------------------------------------------------------------------
# graph-formulation time evolution (energy-conservation pin of U and E)
# ---------------------------------------------------------------------------

def surface_replaced(geom, eta):
    """The geometry with the free surface replaced by the graph zeta_0 = alpha +
    i eta(alpha) (xi = alpha); zeta_0', zeta_0'' by spectral derivatives of eta."""
    M0 = geom.M[0]
    a = TWO_PI * np.arange(M0) / M0
    ea = d_alpha(eta)
    eaa = d_alpha(ea)
    zeta = geom.zeta.copy()
    dzeta = geom.dzeta.copy()
    d2zeta = geom.d2zeta.copy()
    zeta[:M0] = a + 1j * eta
    dzeta[:M0] = 1.0 + 1j * ea
    d2zeta[:M0] = 1j * eaa
    return type(geom)(M=geom.M, zeta=zeta, dzeta=dzeta, d2zeta=d2zeta, zc=geom.zc,
                      ellipses=geom.ellipses)


def graph_rhs(geom, flow, eta, phit, tau=0.1, g=1.0):
    """(eta_t, phi~_t) for xi = alpha: eta_t = s_alpha U (eq. graph:eta:t) and
    eq. phitileq with V = eta_alpha U, C(t) = 0, rho = 1:
      phi~_t = (phi~_alpha/s_alpha) V + (d phi~/dn) U - |grad phi|^2/2 - g eta
               + tau theta_alpha/s_alpha,
      |grad phi|^2 = (phi_alpha/s_alpha)^2 + U^2,  d phi~/dn = U - d phi_mv/dn.
    Obstacles and bottom do not move.  Returns (eta_t, phit_t, omega, geometry)."""
    gs = surface_replaced(geom, eta)
    om, U, _ = solve(gs, flow, phit)
    z0, dz0, d2z0 = gs.block(0)
    ea = dz0.imag
    s = np.sqrt(1.0 + ea * ea)
    V = ea * U
    dPm = dPhi_mv(gs, flow, z0)
    dphimv_dn = np.real(dPm * 1j * dz0) / s
    phit_a = d_alpha(phit)
    phi_a = phit_a + np.real(dPm * dz0)
    grad2 = (phi_a / s) ** 2 + U ** 2
    theta_a = d2z0.imag / (1.0 + ea * ea)
    phit_t = (phit_a / s) * V + (U - dphimv_dn) * U - 0.5 * grad2 - g * eta + tau * theta_a / s
    return s * U, phit_t, om, gs


def evolve_energy(geom, flow, eta0, phit0, dt, nsteps, tau=0.1, g=1.0):
    """Classical RK4 on (eta, phi~); returns the energy of eq. E:formula at each step."""
    eta, phit = eta0.copy(), phit0.copy()
    Es = []
    for n in range(nsteps + 1):
        k1e, k1p, om, gs = graph_rhs(geom, flow, eta, phit, tau, g)
        Es.append(energy(gs, flow, phit, om, tau=tau, g=g))
        if n == nsteps:
            break
        k2e, k2p, _, _ = graph_rhs(geom, flow, eta + 0.5 * dt * k1e, phit + 0.5 * dt * k1p, tau, g)
        k3e, k3p, _, _ = graph_rhs(geom, flow, eta + 0.5 * dt * k2e, phit + 0.5 * dt * k2p, tau, g)
        k4e, k4p, _, _ = graph_rhs(geom, flow, eta + dt * k3e, phit + dt * k3p, tau, g)
        eta = eta + dt / 6.0 * (k1e + 2 * k2e + 2 * k3e + k4e)
        phit = phit + dt / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
    return np.array(Es)


# ---------------------------------------------------------------------------
# auxiliary Dirichlet problem for Phi_t - C(t) (Sec. 4, eq. pressure:d:prob)
# ---------------------------------------------------------------------------

def curvature_surface(geom):
    """kappa = theta_alpha / s_alpha on Gamma_0, theta the tangent angle:
    theta_alpha = Im{zeta'' conj(zeta')}/|zeta'|^2, so
    kappa = Im{zeta'' conj(zeta')} / |zeta'|^3 (positive where the surface is
    concave up; for a graph y = eta(x) this is eta''/(1 + eta'^2)^(3/2), the
    sign of the tau theta_alpha / s_alpha term of eq. phitileq)."""
    _, dz0, d2z0 = geom.block(0)
    return np.imag(d2z0 * np.conj(dz0)) / np.abs(dz0) ** 3


def pressure_rhs(geom, flow, phitilde, U, tau=0.1, g=1.0):
    """b^aux of eq. pressure:d:prob: b_0 = tau kappa - |grad phi|^2/2 - g eta on
    the surface, b_k = 0 on the solid boundaries.  On the surface
    |grad phi|^2 = (phi_alpha / s_alpha)^2 + U^2 (tangential and normal parts),
    phi_alpha from phi~ and the multi-valued part (phi_alpha_surface), U the
    normal velocity of the same state, eta = Im zeta_0."""
    z0, dz0, _ = geom.block(0)
    s = np.abs(dz0)
    phia = phi_alpha_surface(geom, flow, phitilde)
    b = np.zeros(geom.N, dtype=np.float64)
    b[: geom.M[0]] = (tau * curvature_surface(geom) - 0.5 * ((phia / s) ** 2 + U ** 2)
                      - g * z0.imag)
    return b


def solve_aux(geom, flow, phitilde, tau=0.1, g=1.0):
    """omega and U of the state, then omega^aux of A omega^aux = b^aux (the
    same matrix, Sec. 4).  Returns (omega, U, b_aux, omega_aux)."""
    A = assemble(geom)
    omega = solve_dense(A, rhs(geom, flow, phitilde))
    U = normal_velocity(geom, flow, omega)
    b = pressure_rhs(geom, flow, phitilde, U, tau, g)
    return omega, U, b, solve_dense(A, b)


def phi_tilde_at(geom, omega, z):
    """Phi~(z) = sum_j Phi_j(z) at points z of Omega by the trapezoidal rule
    applied to the Cauchy integrals of eq. w123 (the free surface with density
    omega_0, the solid boundaries with i omega_j): accurate for z several node
    spacings away from every boundary."""
    M = list(geom.M)
    o = offsets(M)
    w = split(omega, M)
    z = np.asarray(z, dtype=np.complex128)
    acc = np.zeros(z.shape, dtype=np.complex128)
    for j in range(len(M)):
        zj = geom.zeta[o[j]:o[j + 1]]
        dzj = geom.dzeta[o[j]:o[j + 1]]
        c = 1.0 if j == 0 else 1j
        acc += (half_cot(zj[None, :] - z[:, None]) * dzj[None, :]) @ (c * w[j]) / M[j]
    return acc / 1j


def phi_tilde_boundary(geom, omega):
    """Phi~ on every boundary from the fluid side (Gamma_0^-, Gamma_k^+), per
    boundary, by the Plemelj formula applied to eq. w123 (Sec. 4: the real and
    imaginary parts needed for Phi_t - C on the boundaries).

    Re on Gamma_0 and Im on Gamma_k are the rows of eq. lin:sys (A omega, plus
    the mean of omega_k that the -E_k term removes on obstacles); Im on Gamma_0
    is the psi of the energy (psi_surface without psi_mv).  Re on a solid
    boundary k (the jump (i/2) omega_k is imaginary and drops out):
      Re Phi~(zeta_k(alpha)^+) = (1/M_0) sum_l Im{zeta_0' 1/2 cot((zeta_0 - zeta_k)/2)} omega_0
        + sum_{j >= 1, j != k} (1/M_j) sum_l Re{zeta_j' 1/2 cot((zeta_j - zeta_k)/2)} omega_j
        + (1/M_k) sum_l Greg_kk omega_k - (1/2) H omega_k,
    with Greg_kk(alpha, beta) = Re{zeta_k'(beta) 1/2 cot((zeta_k(beta) - zeta_k(alpha))/2)}
    - 1/2 cot((beta - alpha)/2) (diagonal limit Re{zeta_k''/(2 zeta_k')}, as for
    G_00 in Sec. 3.4) and H the Hilbert transform of symbol -i sgn(k): the
    principal value of the 1/2 cot((beta - alpha)/2) part is -(1/2) H omega_k."""
    M = list(geom.M)
    o = offsets(M)
    w = split(omega, M)
    A = assemble(geom)
    y = A @ omega
    out = []
    zero_flow = SimpleNamespace(V1=0.0, a=np.zeros(max(0, len(M) - 2)))   # psi_mv = 0
    re0 = y[o[0]:o[1]]
    im0 = psi_surface(geom, zero_flow, omega)
    out.append(re0 + 1j * im0)
    for k in range(1, len(M)):
        zk = geom.zeta[o[k]:o[k + 1]]
        dzk = geom.dzeta[o[k]:o[k + 1]]
        d2zk = geom.d2zeta[o[k]:o[k + 1]]
        imk = y[o[k]:o[k + 1]] + (w[k].mean() if k >= 2 else 0.0)
        rek = np.zeros(M[k])
        for j in range(len(M)):
            zj = geom.zeta[o[j]:o[j + 1]]
            dzj = geom.dzeta[o[j]:o[j + 1]]
            if j == k:
                a = TWO_PI * np.arange(M[k]) / M[k]
                with np.errstate(divide="ignore", invalid="ignore"):
                    G = np.real(dzk[None, :] * half_cot(zk[None, :] - zk[:, None])
                                - half_cot(a[None, :] - a[:, None]))
                G[np.arange(M[k]), np.arange(M[k])] = np.real(d2zk / (2.0 * dzk))
                rek += G @ w[k] / M[k] - 0.5 * hilbert(w[k])
            else:
                F = dzj[None, :] * half_cot(zj[None, :] - zk[:, None])
                rek += (F.imag if j == 0 else F.real) @ w[j] / M[j]
        out.append(rek + 1j * imk)
    return out


# ---------------------------------------------------------------------------
# time evolution of the graph formulation (Sec. 2, eqs. graph:eta:t, phitileq)
# ---------------------------------------------------------------------------

def filter36(f):
    """The 36th-order Fourier filter of eq. filter: mode k multiplied by
    exp(-36 (|k|/k_max)^36), k_max = M/2 (for even M the Nyquist mode has
    |k| = k_max)."""
    M = len(f)
    k = np.abs(np.fft.fftfreq(M, d=1.0 / M))
    rho = np.exp(-36.0 * (k / (M / 2.0)) ** 36)
    return np.real(np.fft.ifft(rho * np.fft.fft(f)))


def evolve_graph(geom, flow, eta0, phit0, dt, nsteps, tau=0.1, g=1.0, filt=False):
    """Classical RK4 on (eta, phi~) with the right-hand side of graph_rhs; with
    filt, eq. filter is applied to eta and phi~ at the end of every step (not
    in the stages).  Returns (eta, phi~, energies at t = 0, dt, ..., nsteps dt)."""
    eta, phit = eta0.copy(), phit0.copy()
    Es = []
    for n in range(nsteps + 1):
        k1e, k1p, om, gs = graph_rhs(geom, flow, eta, phit, tau, g)
        Es.append(energy(gs, flow, phit, om, tau=tau, g=g))
        if n == nsteps:
            break
        k2e, k2p, _, _ = graph_rhs(geom, flow, eta + 0.5 * dt * k1e, phit + 0.5 * dt * k1p, tau, g)
        k3e, k3p, _, _ = graph_rhs(geom, flow, eta + 0.5 * dt * k2e, phit + 0.5 * dt * k2p, tau, g)
        k4e, k4p, _, _ = graph_rhs(geom, flow, eta + dt * k3e, phit + dt * k3p, tau, g)
        eta = eta + dt / 6.0 * (k1e + 2 * k2e + 2 * k3e + k4e)
        phit = phit + dt / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
        if filt:
            eta, phit = filter36(eta), filter36(phit)
    return eta, phit, np.array(Es)


# ---------------------------------------------------------------------------
# App. B: psi prescribed on the solid boundaries, circulations a_j unknown
# ---------------------------------------------------------------------------

def phi_cyl(z):
    """Re Phi_cyl(z) = arg(1 - e^{iz}), Phi_cyl(z) = -i log(1 - e^{iz}) (principal
    branch; Im Phi_cyl = psi_cyl and Phi_cyl' matches eq. d:phi:cyl).  Used above
    the obstacle centre, where |e^{iz}| < 1 keeps the branch continuous."""
    return np.angle(1.0 - np.exp(1j * z))


def assemble_alt(geom):
    """The operator of eq. A:alt: B + sum_{m>=2} u_m <1_m, .>, where u_m holds
    phi_cyl(zeta_0 - z_m) on the surface rows and psi_cyl(zeta_k - z_m) on the
    solid rows, and <1_m, w> is the mean of w over boundary m."""
    M = list(geom.M)
    o = offsets(M)
    bid = block_ids(M)
    rows = np.arange(geom.N)
    # B: the Table 1 entries / M_j and the +-1/2 diagonal (no -E_k term)
    zt = geom.zeta[:, None]
    zs = geom.zeta[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        F = geom.dzeta[None, :] * half_cot(zs - zt)
    kr = bid[:, None]
    js = bid[None, :]
    B = np.where((kr == 0) & (js == 0), F.imag,
        np.where(kr == 0, F.real,
        np.where(js == 0, -F.real, F.imag)))
    B[rows, rows] = (geom.d2zeta / (2.0 * geom.dzeta)).imag
    B = B / np.asarray(M, dtype=np.float64)[bid][None, :]
    B[rows, rows] += np.where(bid == 0, -0.5, 0.5)
    A = B
    for m in range(2, len(M)):
        d = geom.zeta - geom.zc[m - 2]
        u = np.where(bid == 0, phi_cyl(d), psi_cyl(d))
        A[:, o[m]:o[m + 1]] += u[:, None] / M[m]
    return A


def rhs_alt(geom, V1, phic, psi_solid):
    """b_0 = phi - V1 xi (given as phic on the surface), b_k = psi - V1 eta_k on
    the solid nodes (psi_solid given there), App. B."""
    b = np.empty(geom.N)
    M0 = geom.M[0]
    b[:M0] = phic
    b[M0:] = psi_solid - V1 * geom.zeta[M0:].imag
    return b


def solve_alt(geom, V1, phic, psi_solid):
    """(omega, U, a): the App. B solve; a_j = <1_j, omega> are the circulations
    and U is the normal velocity of Phi = Phi~ + sum a_j Phi_cyl(z - z_j) + V1 z."""
    A = assemble_alt(geom)
    omega = solve_dense(A, rhs_alt(geom, V1, phic, psi_solid))
    a = psi_k(geom, omega)
    U = normal_velocity(geom, type("F", (), {"V1": V1, "a": a})(), omega)
    return omega, U, a


# ---------------------------------------------------------------------------
# HLS (angle-arclength) formulation with P theta reconstruction (Sec. 2,
# eqs. za:zt, theta:t, definitionOfV, CS:th, xi:eta:recon, Pth:t)
# ---------------------------------------------------------------------------

def antiderivative(f):
    """Zero-mean spectral antiderivative of a periodic sample vector: symbol
    1/(ik) for k != 0, 0 for k = 0 (and the Nyquist mode, as for d_alpha)."""
    k = wavenumbers(len(f))
    F = np.fft.fft(f)
    G = np.zeros_like(F)
    nz = k != 0
    G[nz] = F[nz] / (1j * k[nz])
    return np.real(np.fft.ifft(G))


def hls_curve(Ptheta):
    """Curve from P theta (eq. CS:th, eq. xi:eta:recon): C = P0[cos P theta],
    S = P0[sin P theta], P0 theta = arg(C - iS), s_alpha = (C^2 + S^2)^(-1/2),
    zeta_alpha = s_alpha e^{i theta}; xi = alpha + xi_aux - xi_aux(0),
    eta = eta_aux - P0[eta_aux xi_alpha] with xi_aux, eta_aux the zero-mean
    antiderivatives of xi_alpha - 1 and eta_alpha.  Returns (zeta, zeta',
    zeta'', theta, s_alpha); zeta'' = i theta_alpha zeta' (s_alpha is constant)."""
    M = len(Ptheta)
    a = TWO_PI * np.arange(M) / M
    C = np.mean(np.cos(Ptheta))
    S = np.mean(np.sin(Ptheta))
    P0th = np.angle(C - 1j * S)
    theta = Ptheta + P0th
    s = (C * C + S * S) ** -0.5
    dz = s * np.exp(1j * theta)
    xi_aux = antiderivative(dz.real - 1.0)
    eta_aux = antiderivative(dz.imag)
    xi = a + xi_aux - xi_aux[0]
    eta = eta_aux - np.mean(eta_aux * dz.real)
    d2z = 1j * d_alpha(Ptheta) * dz
    return xi + 1j * eta, dz, d2z, theta, s


def hls_surface_replaced(geom, Ptheta):
    z, dz, d2z, _, _ = hls_curve(Ptheta)
    M0 = geom.M[0]
    zeta, dzeta, d2zeta = geom.zeta.copy(), geom.dzeta.copy(), geom.d2zeta.copy()
    zeta[:M0], dzeta[:M0], d2zeta[:M0] = z, dz, d2z
    return type(geom)(M=geom.M, zeta=zeta, dzeta=dzeta, d2zeta=d2zeta, zc=geom.zc,
                      ellipses=geom.ellipses)


def hls_tangential_velocity(theta_a, U, dz0):
    """V of eq. definitionOfV: zero-mean antiderivative of theta_alpha U -
    P0[theta_alpha U], shifted so that V(0) = U(0) eta_alpha(0)/xi_alpha(0)
    (keeps xi(0) = 0)."""
    V = antiderivative(theta_a * U - np.mean(theta_a * U))
    return V - V[0] + U[0] * dz0[0].imag / dz0[0].real


def hls_theta_t(U, V, theta_a, s):
    """(P theta)_t = P[(U_alpha + V theta_alpha)/s_alpha] (eqs. theta:t, Pth:t)."""
    th_t = (d_alpha(U) + V * theta_a) / s
    return th_t - np.mean(th_t)


def hls_rhs(geom, flow, Ptheta, phit, tau=0.1, g=1.0):
    """((P theta)_t, phi~_t) of the HLS formulation with the velocity-potential
    solve: V from eq. definitionOfV, V_alpha = theta_alpha U - P0[theta_alpha U],
    its constant fixed by xi(0) = 0, i.e. V(0) = U(0) eta_alpha(0)/xi_alpha(0);
    (P theta)_t = P[(U_alpha + V theta_alpha)/s_alpha] (eq. Pth:t); phi~_t by
    eq. phitileq with C(t) = 0, rho = 1.  Returns (Ptheta_t, phit_t, omega, geometry)."""
    gs = hls_surface_replaced(geom, Ptheta)
    om, U, _ = solve(gs, flow, phit)
    z0, dz0, _ = gs.block(0)
    s = np.abs(dz0)
    theta_a = d_alpha(Ptheta)
    V = hls_tangential_velocity(theta_a, U, dz0)
    th_t = hls_theta_t(U, V, theta_a, s)
    dPm = dPhi_mv(gs, flow, z0)
    dphimv_dn = np.real(dPm * 1j * dz0) / s
    phit_a = d_alpha(phit)
    phi_a = phit_a + np.real(dPm * dz0)
    grad2 = (phi_a / s) ** 2 + U ** 2
    phit_t = (phit_a / s) * V + (U - dphimv_dn) * U - 0.5 * grad2 - g * z0.imag + tau * theta_a / s
    return th_t, phit_t, om, gs


def evolve_hls(geom, flow, Ptheta0, phit0, dt, nsteps, tau=0.1, g=1.0, filt=False):
    """Classical RK4 on (P theta, phi~) with hls_rhs; eq. filter on both at the
    end of each step when filt.  Returns (P theta, phi~, energies)."""
    th, ph = Ptheta0.copy(), phit0.copy()
    Es = []
    for n in range(nsteps + 1):
        k1t, k1p, om, gs = hls_rhs(geom, flow, th, ph, tau, g)
        Es.append(energy(gs, flow, ph, om, tau=tau, g=g))
        if n == nsteps:
            break
        k2t, k2p, _, _ = hls_rhs(geom, flow, th + 0.5 * dt * k1t, ph + 0.5 * dt * k1p, tau, g)
        k3t, k3p, _, _ = hls_rhs(geom, flow, th + 0.5 * dt * k2t, ph + 0.5 * dt * k2p, tau, g)
        k4t, k4p, _, _ = hls_rhs(geom, flow, th + dt * k3t, ph + dt * k3p, tau, g)
        th = th + dt / 6.0 * (k1t + 2 * k2t + 2 * k3t + k4t)
        ph = ph + dt / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
        if filt:
            th, ph = filter36(th), filter36(ph)
    return th, ph, np.array(Es)


# ---------------------------------------------------------------------------
# an eighth-order explicit step: Gragg-Bulirsch-Stoer extrapolation
# ---------------------------------------------------------------------------

GBS_SEQUENCE = (2, 4, 6, 8)


def gbs8_step(f, y, h):
    """One step of size h of y' = f(y): the explicit midpoint rule with n
    substeps, z_0 = y, z_1 = z_0 + (h/n) f(z_0), z_{m+1} = z_{m-1} + 2 (h/n) f(z_m),
    T_n = z_n, for n = 2, 4, 6, 8, then Aitken-Neville extrapolation in
    (h/n)^2 to h -> 0: T_{j,k} = T_{j,k-1} + (T_{j,k-1} - T_{j-1,k-1}) /
    ((n_j/n_{j-k})^2 - 1).  Gragg's expansion of the midpoint rule (even n)
    has only even powers of h/n, so four levels give order 8."""
    f0 = f(y)
    T = []
    for n in GBS_SEQUENCE:
        hs = h / n
        zm, z = y, y + hs * f0
        for _ in range(1, n):
            zm, z = z, zm + 2.0 * hs * f(z)
        row = [z]
        for k in range(1, len(T) + 1):
            r = (n / GBS_SEQUENCE[len(T) - k]) ** 2
            row.append(row[k - 1] + (row[k - 1] - T[-1][k - 1]) / (r - 1.0))
        T.append(row)
    return T[-1][-1]


def evolve_explicit(geom, flow, y1_0, phit0, dt, nsteps, step, tau=0.1, g=1.0, filt=False,
                    formulation="graph"):
    """(eta, phi~) (formulation "graph") or (P theta, phi~) ("hls") advanced
    by nsteps of a one-step method step(f, y, h), the filter after each step
    when filt.  Returns (first variable, phi~, energies at t = 0, dt, ...,
    nsteps dt)."""
    M0 = geom.M[0]
    rhs = graph_rhs if formulation == "graph" else hls_rhs

    def f(y):
        a, b, _, _ = rhs(geom, flow, y[:M0], y[M0:], tau, g)
        return np.concatenate([a, b])

    y = np.concatenate([y1_0, phit0])
    Es = []
    for n in range(nsteps + 1):
        _, _, om, gs = rhs(geom, flow, y[:M0], y[M0:], tau, g)
        Es.append(energy(gs, flow, y[M0:], om, tau=tau, g=g))
        if n == nsteps:
            break
        y = step(f, y, dt)
        if filt:
            y = np.concatenate([filter36(y[:M0]), filter36(y[M0:])])
    return y[:M0], y[M0:], np.array(Es)


def evolve_gbs8(geom, flow, y1_0, phit0, dt, nsteps, tau=0.1, g=1.0, filt=False,
                formulation="graph"):
    """evolve_explicit with gbs8_step."""
    return evolve_explicit(geom, flow, y1_0, phit0, dt, nsteps, gbs8_step, tau, g, filt,
                           formulation)


# ---------------------------------------------------------------------------
# the paper's time integrator: eighth-order Dormand-Prince (Sec. 7.1)
# ---------------------------------------------------------------------------
#
# Sec. 7.1 steps every problem with the eighth-order Dormand-Prince
# Runge-Kutta scheme of Hairer, Norsett & Wanner (Solving Ordinary
# Differential Equations I, Sec. II.10: the 12-stage method DOP853), at a
# fixed step dt = Delta t / d; Sec. 7.4 counts 12 solves per step.  Below is
# its published Butcher tableau, written out as the publication gives it:
# c_i = sum_j a_ij, with c_4 = (6 - sqrt 6)/30, c_3 = (2/3) c_4,
# c_2 = (2/3) c_3 and c_5 = (6 + sqrt 6)/30.

DP8_C = np.array([
    0.0, 0.526001519587677318785587544488e-01, 0.789002279381515978178381316732e-01,
    0.118350341907227396726757197510e+00, 0.281649658092772603273242802490e+00,
    1.0 / 3.0, 0.25, 4.0 / 13.0, 127.0 / 195.0, 0.6, 6.0 / 7.0, 1.0])

DP8_A = np.zeros((12, 12))
DP8_A[1, :1] = [5.26001519587677318785587544488e-2]
DP8_A[2, :2] = [1.97250569845378994544595329183e-2, 5.91751709536136983633785987549e-2]
DP8_A[3, :3] = [2.95875854768068491816892993775e-2, 0.0, 8.87627564304205475450678981324e-2]
DP8_A[4, :4] = [2.41365134159266685502369798665e-1, 0.0, -8.84549479328286085344864962717e-1,
                9.24834003261792003115737966543e-1]
DP8_A[5, :5] = [3.7037037037037037037037037037e-2, 0.0, 0.0, 1.70828608729473871279604482173e-1,
                1.25467687566822425016691814123e-1]
DP8_A[6, :6] = [3.7109375e-2, 0.0, 0.0, 1.70252211019544039314978060272e-1,
                6.02165389804559606850219397283e-2, -1.7578125e-2]
DP8_A[7, :7] = [3.70920001185047927108779319836e-2, 0.0, 0.0, 1.70383925712239993810214054705e-1,
                1.07262030446373284651809199168e-1, -1.53194377486244017527936158236e-2,
                8.27378916381402288758473766002e-3]
DP8_A[8, :8] = [6.24110958716075717114429577812e-1, 0.0, 0.0, -3.36089262944694129406857109825e0,
                -8.68219346841726006818189891453e-1, 2.75920996994467083049415600797e1,
                2.01540675504778934086186788979e1, -4.34898841810699588477366255144e1]
DP8_A[9, :9] = [4.77662536438264365890433908527e-1, 0.0, 0.0, -2.48811461997166764192642586468e0,
                -5.90290826836842996371446475743e-1, 2.12300514481811942347288949897e1,
                1.52792336328824235832596922938e1, -3.32882109689848629194453265587e1,
                -2.03312017085086261358222928593e-2]
DP8_A[10, :10] = [-9.3714243008598732571704021658e-1, 0.0, 0.0, 5.18637242884406370830023853209e0,
                  1.09143734899672957818500254654e0, -8.14978701074692612513997267357e0,
                  -1.85200656599969598641566180701e1, 2.27394870993505042818970056734e1,
                  2.49360555267965238987089396762e0, -3.0467644718982195003823669022e0]
DP8_A[11, :11] = [2.27331014751653820792359768449e0, 0.0, 0.0, -1.05344954667372501984066689879e1,
                  -2.00087205822486249909675718444e0, -1.79589318631187989172765950534e1,
                  2.79488845294199600508499808837e1, -2.85899827713502369474065508674e0,
                  -8.87285693353062954433549289258e0, 1.23605671757943030647266201528e1,
                  6.43392746015763530355970484046e-1]

DP8_B = np.array([
    5.42937341165687622380535766363e-2, 0.0, 0.0, 0.0, 0.0, 4.45031289275240888144113950566e0,
    1.89151789931450038304281599044e0, -5.8012039600105847814672114227e0,
    3.1116436695781989440891606237e-1, -1.52160949662516078556178806805e-1,
    2.01365400804030348374776537501e-1, 4.47106157277725905176885569043e-2])


def dp8_step(f, y, h):
    """One step of size h of y' = f(y) (autonomous) with the tableau above:
    k_i = f(y + h sum_{j<i} a_ij k_j), i = 1..12, then y + h sum_i b_i k_i."""
    k = []
    for i in range(12):
        yi = y.copy()
        for j in range(i):
            if DP8_A[i, j] != 0.0:
                yi = yi + h * DP8_A[i, j] * k[j]
        k.append(f(yi))
    out = y.copy()
    for i in range(12):
        if DP8_B[i] != 0.0:
            out = out + h * DP8_B[i] * k[i]
    return out


def evolve_dp8(geom, flow, y1_0, phit0, dt, nsteps, tau=0.1, g=1.0, filt=False,
               formulation="graph"):
    """evolve_explicit with dp8_step: the paper's fixed-step time stepping."""
    return evolve_explicit(geom, flow, y1_0, phit0, dt, nsteps, dp8_step, tau, g, filt,
                           formulation)


# ---------------------------------------------------------------------------
# vortex-sheet evolution: gamma_0,t from eqs. gam:t:final and gam:t:aux (Sec. 4)
# ---------------------------------------------------------------------------

def gamma_t_matrix(geom):
    """The operator of eqs. gam:t:final and gam:t:aux on (gamma_0,t, ...,
    gamma_N,t): surface rows (1/2 I + K_00^*) and -G_j0^*; solid rows k G_0k^*,
    -1/2 I + K_kk^* and K_jk^* (starred operators as in eq. lin:sys2, weights
    1/M_j, eq. KG:tmat)."""
    M = list(geom.M)
    o = offsets(M)
    nb = len(M)
    T = np.zeros((geom.N, geom.N))
    for k in range(nb):
        rk = slice(o[k], o[k + 1])
        for j in range(nb):
            cj = slice(o[j], o[j + 1])
            c = vs_kernel_block(geom, j, k) / M[j]
            if k == 0:
                T[rk, cj] = c.imag if j == 0 else -c.real
            else:
                T[rk, cj] = c.real if j == 0 else c.imag
        T[rk, rk] += (0.5 if k == 0 else -0.5) * np.eye(M[k])
    return T


def surface_source_sums(geom, x):
    """For every node m (any boundary k) the Table 1 sums over the surface
    sources l with density x: S[m] = (1/M_0) sum_l zeta_0'(beta_l)/2
    cot((zeta_0(beta_l) - zeta_k(alpha_m))/2) x_l; on the surface the real
    part is regularised by -1/2 cot((beta_l - alpha_m)/2) and the diagonal
    term is zeta''/(2 zeta') (the limits of K_00 and G_00)."""
    M = list(geom.M)
    M0 = M[0]
    z0, dz0, d2z0 = geom.block(0)
    with np.errstate(divide="ignore", invalid="ignore"):
        F = dz0[None, :] * half_cot(z0[None, :] - geom.zeta[:, None])
    a0 = TWO_PI * np.arange(M0) / M0
    with np.errstate(divide="ignore", invalid="ignore"):
        F[:M0] = F[:M0] - half_cot(a0[None, :] - a0[:, None])
    F[np.arange(M0), np.arange(M0)] = d2z0 / (2.0 * dz0)
    return F @ x / M0


def antiderivative_blocks(geom, v):
    return np.concatenate([antiderivative(b) for b in split(v, geom.M)])


def vs_surface_W(fb, gamma0, s, t):
    """W = grad phi - gamma_0/(2 s_alpha) t (eq. dphi:W:gam); fb = u - i v."""
    return fb.real - gamma0 / (2 * s) * t.real, -fb.imag - gamma0 / (2 * s) * t.imag


def vs_bernoulli(Wx, Wy, t, V, gamma0, s, forcing, F00):
    """The bracket of eq. gam:t:final: -W.W/2 + (V - W.t) gamma_0/(2 s_alpha)
    - gamma_0^2/(8 s_alpha^2) + (tau theta_alpha/s_alpha - g eta) - F_00 gamma_0."""
    WW = Wx * Wx + Wy * Wy
    Wt = Wx * t.real + Wy * t.imag
    return -0.5 * WW + (V - Wt) * gamma0 / (2 * s) - gamma0 ** 2 / (8 * s * s) + forcing - F00


def vs_graph_rhs(geom, flow, eta, gamma0, tau=0.1, g=1.0):
    """(eta_t, gamma_0,t) of the vortex-sheet formulation with xi = alpha (Sec. 4):
    U and gamma_1..N from eq. lin:sys2; V = eta_alpha U; W = grad phi -
    gamma_0/(2 s_alpha) t (eq. dphi:W:gam) with grad phi on the surface from the
    Cauchy integrals of omega_0 = -d^-1 gamma_0, omega_j = d^-1 gamma_j (zero-mean
    antiderivatives); F_00, F_k0 of eq. Fk:from:UV; right-hand sides of eqs.
    gam:t:final (surface) and gam:t:aux (solids); then the solve with
    gamma_t_matrix.  Returns (eta_t, gamma0_t, U, geometry)."""
    gs = surface_replaced(geom, eta)
    M = list(gs.M)
    M0 = M[0]
    U, gam = vs_solve(gs, flow, gamma0)
    z0, dz0, d2z0 = gs.block(0)
    s = np.abs(dz0)
    ea = dz0.imag
    V = ea * U
    gall = np.concatenate([gamma0] + list(gam))
    om = antiderivative_blocks(gs, gall)
    om[:M0] = -om[:M0]
    fb = boundary_dphi(gs, flow, om)[0]                 # u - i v on the surface (fluid side)
    t = dz0 / s
    Wx, Wy = vs_surface_W(fb, gamma0, s, t)
    x1 = V * gamma0 / s
    x2 = U * gamma0 / s
    S1 = surface_source_sums(gs, x1)
    S2 = surface_source_sums(gs, x2)
    F00 = -0.5 * hilbert(x2) + S1[:M0].imag + S2[:M0].real
    Fk0 = S1[M0:].real - S2[M0:].imag
    theta_a = d2z0.imag / (1.0 + ea * ea)
    Q = vs_bernoulli(Wx, Wy, t, V, gamma0, s, tau * theta_a / s - g * z0.imag, F00)
    r = np.empty(gs.N)
    r[:M0] = d_alpha(Q)
    r[M0:] = -np.concatenate([d_alpha(b) for b in split(Fk0, M[1:])])
    gt = np.linalg.solve(gamma_t_matrix(gs), r)
    return s * U, gt[:M0], U, gs


def evolve_vs_graph(geom, flow, eta0, gamma00, dt, nsteps, tau=0.1, g=1.0, step=None):
    """Classical RK4 on (eta, gamma_0) with vs_graph_rhs, or the one-step
    method step(f, y, h) (e.g. dp8_step) when given.  Returns (eta, gamma_0)."""
    if step is not None:
        M0 = geom.M[0]

        def f(y):
            a, b, _, _ = vs_graph_rhs(geom, flow, y[:M0], y[M0:], tau, g)
            return np.concatenate([a, b])

        y = np.concatenate([eta0, gamma00])
        for _ in range(nsteps):
            y = step(f, y, dt)
        return y[:M0], y[M0:]
    eta, gm = eta0.copy(), gamma00.copy()
    for _ in range(nsteps):
        k1e, k1g, _, _ = vs_graph_rhs(geom, flow, eta, gm, tau, g)
        k2e, k2g, _, _ = vs_graph_rhs(geom, flow, eta + 0.5 * dt * k1e, gm + 0.5 * dt * k1g, tau, g)
        k3e, k3g, _, _ = vs_graph_rhs(geom, flow, eta + 0.5 * dt * k2e, gm + 0.5 * dt * k2g, tau, g)
        k4e, k4g, _, _ = vs_graph_rhs(geom, flow, eta + dt * k3e, gm + dt * k3g, tau, g)
        eta = eta + dt / 6.0 * (k1e + 2 * k2e + 2 * k3e + k4e)
        gm = gm + dt / 6.0 * (k1g + 2 * k2g + 2 * k3g + k4g)
    return eta, gm
