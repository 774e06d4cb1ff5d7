"""Seeded synthetic initial conditions (host, FP64).

These generators produce the input data for the CPU oracle and the CUDA
library alike.  They hold none of the step's arithmetic: they only build
conserved cell averages (rho, M, E) and face-averaged magnetic fields from
analytic or random fields.  Face fields come from edge integrals of a vector
potential, so the discrete divergence of every initial state is zero to
round-off (the vector-potential set-up of the paper's problem scripts,
Sec. 3.4).

Array shapes follow the library interface:
  cons[5][nz][ny][nx], b1[nz][ny][nx+1], b2[nz][ny+1][nx], b3[nz+1][ny][nx].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CART, SPH = 0, 1
PERIODIC, OUTFLOW = 0, 1

# Gauss-Legendre nodes for the edge integrals of the vector potential.  The
# discrete divergence of the face field is zero for any order (each edge
# integral is shared by the faces around it); the order only sets how well
# the face averages match the analytic curl.
_GL = {q: np.polynomial.legendre.leggauss(q) for q in (2, 3, 4, 6)}
_GL_X, _GL_W = _GL[6]


@dataclass
class Block:
    """One mesh block: sizes, coordinate system, extents, boundary kinds."""
    n: tuple          # (nx, ny, nz)
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    coord: int = CART
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)

    def faces(self, d):
        return np.linspace(self.lo[d], self.hi[d], self.n[d] + 1)

    def centers(self, d):
        f = self.faces(d)
        return 0.5 * (f[1:] + f[:-1])


@dataclass
class InitialState:
    block: Block
    cons: np.ndarray
    b1: np.ndarray
    b2: np.ndarray
    b3: np.ndarray
    gamma: float
    meta: dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# geometry of the generator (face areas and edge element lengths)
# ---------------------------------------------------------------------------

def _face_areas(b: Block):
    f = [b.faces(d) for d in range(3)]
    nx, ny, nz = b.n
    if b.coord == CART:
        dx = [(b.hi[d] - b.lo[d]) / b.n[d] for d in range(3)]
        return (np.full((nz, ny, nx + 1), dx[1] * dx[2]),
                np.full((nz, ny + 1, nx), dx[0] * dx[2]),
                np.full((nz + 1, ny, nx), dx[0] * dx[1]))
    r, t = f[0], f[1]
    dphi = (b.hi[2] - b.lo[2]) / nz
    a1 = (r[None, None, :] ** 2 * (np.cos(t[:-1]) - np.cos(t[1:]))[None, :, None] * dphi)
    a1 = np.broadcast_to(a1, (nz, ny, nx + 1)).copy()
    a2 = (0.5 * (r[1:] ** 2 - r[:-1] ** 2)[None, None, :] * np.sin(t)[None, :, None] * dphi)
    a2 = np.broadcast_to(a2, (nz, ny + 1, nx)).copy()
    a3 = 0.5 * (r[1:] ** 2 - r[:-1] ** 2)[None, None, :] * (t[1:] - t[:-1])[None, :, None]
    a3 = np.broadcast_to(a3, (nz + 1, ny, nx)).copy()
    return a1, a2, a3


def _edge_integrals(b: Block, A, gl=6):
    """Line integrals of the vector potential A(x1, x2, x3) -> (A1, A2, A3)
    (physical components) along every cell edge (Gauss-Legendre order gl)."""
    glx, glw = _GL[gl]
    f = [b.faces(d) for d in range(3)]
    sph = b.coord == SPH

    def along(d):
        # integral of A_d along edges parallel to axis d
        e1, e2 = [q for q in range(3) if q != d]
        xs = f[d]
        mids = 0.5 * (xs[1:] + xs[:-1])
        half = 0.5 * (xs[1:] - xs[:-1])
        pts = mids[:, None] + half[:, None] * glx[None, :]         # (n_d, q)
        wts = half[:, None] * glw[None, :]
        grids = [None, None, None]
        grids[d] = pts[:, :, None, None]
        grids[e1] = f[e1][None, None, :, None]
        grids[e2] = f[e2][None, None, None, :]
        X = [np.broadcast_to(g, (pts.shape[0], pts.shape[1], f[e1].size, f[e2].size))
             for g in grids]
        comp = A(X[0], X[1], X[2])[d]
        comp = np.broadcast_to(comp, X[0].shape)
        if sph:
            if d == 1:
                comp = comp * X[0]                     # r dtheta
            elif d == 2:
                comp = comp * X[0] * np.sin(X[1])      # r sin(theta) dphi
        val = (comp * wts[:, :, None, None]).sum(axis=1)   # (n_d, n_e1, n_e2)
        # reorder to [x3][x2][x1]
        order = {d: 0, e1: 1, e2: 2}
        return np.transpose(val, (order[2], order[1], order[0]))

    return along(0), along(1), along(2)


def face_field_from_potential(b: Block, A, B0=(0.0, 0.0, 0.0), gl=6):
    """Face-averaged B = B0 + curl A from Stokes' theorem on each face."""
    I1, I2, I3 = _edge_integrals(b, A, gl)
    a1, a2, a3 = _face_areas(b)
    b1 = (I3[:, 1:, :] - I3[:, :-1, :] - (I2[1:, :, :] - I2[:-1, :, :])) / a1
    b2 = (I1[1:, :, :] - I1[:-1, :, :] - (I3[:, :, 1:] - I3[:, :, :-1])) / a2
    b3 = (I2[:, :, 1:] - I2[:, :, :-1] - (I1[:, 1:, :] - I1[:, :-1, :])) / a3
    return (np.ascontiguousarray(b1 + B0[0]), np.ascontiguousarray(b2 + B0[1]),
            np.ascontiguousarray(b3 + B0[2]))


def _assemble(b: Block, gamma, rho, v, p, b1, b2, b3, meta=None) -> InitialState:
    """Conserved cell data from cell primitives; E uses the cell-centred
    field taken as the mean of the two bounding faces."""
    bc = (0.5 * (b1[:, :, 1:] + b1[:, :, :-1]), 0.5 * (b2[:, 1:, :] + b2[:, :-1, :]),
          0.5 * (b3[1:, :, :] + b3[:-1, :, :]))
    cons = np.empty((5,) + rho.shape)
    cons[0] = rho
    for d in range(3):
        cons[1 + d] = rho * v[d]
    cons[4] = (p / (gamma - 1.0) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
               + 0.5 * (bc[0] ** 2 + bc[1] ** 2 + bc[2] ** 2))
    return InitialState(b, cons, np.ascontiguousarray(b1), np.ascontiguousarray(b2),
                        np.ascontiguousarray(b3), gamma, meta or {})


def _cell_mesh(b: Block):
    xc = [b.centers(d) for d in range(3)]
    Z, Y, X = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    return X, Y, Z


# ---------------------------------------------------------------------------
# 3D linear fast magnetosonic wave along the grid diagonal (32^3 config)
# ---------------------------------------------------------------------------

def _mhd_primitive_jacobian(gamma, rho, u, v, w, p, bn, bt1, bt2):
    """A(W) of dW/dt + A dW/dx = 0 for W = (rho, u, v, w, p, Bt1, Bt2) with a
    constant normal field (1-D ideal MHD, Sec. 2.1)."""
    A = np.zeros((7, 7))
    A[0, 0] = u; A[0, 1] = rho
    A[1, 1] = u; A[1, 4] = 1 / rho; A[1, 5] = bt1 / rho; A[1, 6] = bt2 / rho
    A[2, 2] = u; A[2, 5] = -bn / rho
    A[3, 3] = u; A[3, 6] = -bn / rho
    A[4, 1] = gamma * p; A[4, 4] = u
    A[5, 1] = bt1; A[5, 2] = -bn; A[5, 5] = u
    A[6, 1] = bt2; A[6, 3] = -bn; A[6, 6] = u
    return A


def fast_eigenvector(gamma=5.0 / 3.0, rho=1.0, p=None, bn=1.0, bt1=math.sqrt(2.0), bt2=0.5):
    """Right-moving fast eigenvector (eigenvalue, vector normalised to
    drho = 1) of the primitive-variable Jacobian at rest."""
    if p is None:
        p = 1.0 / gamma
    A = _mhd_primitive_jacobian(gamma, rho, 0.0, 0.0, 0.0, p, bn, bt1, bt2)
    lam, R = np.linalg.eig(A)
    idx = int(np.argmax(lam.real))
    r = R[:, idx].real
    return float(lam[idx].real), r / r[0]


def diagonal_frame():
    """Orthonormal frame (k_hat, t1, t2) with k_hat along (1,1,1)."""
    k = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    t1 = np.array([-1.0, 1.0, 0.0]) / math.sqrt(2.0)
    t2 = np.cross(k, t1)
    return k, t1, t2


def linear_fast_wave(n=32, amp=1e-6, gamma=5.0 / 3.0) -> InitialState:
    """Periodic unit cube, rho=1, P=1/gamma, B=(1, sqrt2, 0.5) in the wave
    frame rotated so the wave vector is 2*pi*(1,1,1); one right-moving fast
    eigenmode of amplitude amp.  Cell averages are exact."""
    b = Block((n, n, n))
    khat, t1, t2 = diagonal_frame()
    kvec = 2 * math.pi * np.array([1.0, 1.0, 1.0])
    bpar, bt1, bt2 = 1.0, math.sqrt(2.0), 0.5
    B0 = bpar * khat + bt1 * t1 + bt2 * t2
    p0 = 1.0 / gamma
    lam, r = fast_eigenvector(gamma, 1.0, p0, bpar, bt1, bt2)
    X, Y, Z = _cell_mesh(b)
    h = 1.0 / n
    # exact cell average of cos(k.x) over a cube cell
    sinc = np.prod([math.sin(kk * h / 2) / (kk * h / 2) for kk in kvec])
    phase = kvec[0] * X + kvec[1] * Y + kvec[2] * Z
    cavg = np.cos(phase) * sinc
    drho = amp * r[0]
    dv = amp * (r[1] * khat + r[2] * t1 + r[3] * t2)
    dp = amp * r[4]
    db = amp * (r[5] * t1 + r[6] * t2)            # perpendicular to k
    kk2 = float(kvec @ kvec)
    avec = -np.cross(kvec, db) / kk2              # curl(a sin(k.x)) = db cos(k.x)

    def A(x1, x2, x3):
        s = np.sin(kvec[0] * x1 + kvec[1] * x2 + kvec[2] * x3)
        return (avec[0] * s, avec[1] * s, avec[2] * s)

    b1, b2, b3 = face_field_from_potential(b, A, B0)
    # linearised conserved perturbation (first order in amp)
    rho = 1.0 + drho * cavg
    mom = [dv[d] * cavg for d in range(3)]
    bc = (0.5 * (b1[:, :, 1:] + b1[:, :, :-1]), 0.5 * (b2[:, 1:, :] + b2[:, :-1, :]),
          0.5 * (b3[1:, :, :] + b3[:-1, :, :]))
    e = (p0 + dp * cavg) / (gamma - 1.0) + 0.5 * (bc[0] ** 2 + bc[1] ** 2 + bc[2] ** 2)
    cons = np.stack([rho, mom[0], mom[1], mom[2], e])
    period = (1.0 / math.sqrt(3.0)) / lam
    return InitialState(b, cons, b1, b2, b3, gamma,
                        {"speed": lam, "period": period, "amp": amp, "B0": B0})


def linear_wave_box(shape=(512, 512, 256), lengths=(2.0, 2.0, 1.0), amp=1e-6,
                    gamma=5.0 / 3.0, mhd=True, gl=2) -> InitialState:
    """The 3-D linear-wave throughput problem (paper Sec. 6.1) on a periodic
    box of uniform spacing: rho = 1, P = 1/gamma, one right-moving fast
    (MHD, B = (1, sqrt2, 0.5) in the wave frame) or sound (hydro) eigenmode
    of amplitude amp with wave vector 2 pi (1/Lx, 1/Ly, 1/Lz), periodic on
    every axis (along (1,1,2) for the default 2 x 2 x 1 box).  Cell averages
    of the perturbation are exact (one sinc factor per axis); face B comes
    from edge integrals of a vector potential (Gauss-Legendre order gl), so
    div B = 0 to round-off whatever gl."""
    b = Block(tuple(shape), hi=tuple(float(x) for x in lengths))
    kvec = 2 * math.pi * np.array([1.0 / lengths[0], 1.0 / lengths[1], 1.0 / lengths[2]])
    khat = kvec / np.linalg.norm(kvec)
    t1 = np.array([-khat[1], khat[0], 0.0]); t1 /= np.linalg.norm(t1)
    t2 = np.cross(khat, t1)
    bpar, bt1, bt2 = (1.0, math.sqrt(2.0), 0.5) if mhd else (0.0, 0.0, 0.0)
    B0 = bpar * khat + bt1 * t1 + bt2 * t2
    p0 = 1.0 / gamma
    lam, r = fast_eigenvector(gamma, 1.0, p0, bpar, bt1, bt2)
    X, Y, Z = _cell_mesh(b)
    h = [lengths[d] / shape[d] for d in range(3)]
    sinc = np.prod([math.sin(kvec[d] * h[d] / 2) / (kvec[d] * h[d] / 2) for d in range(3)])
    cavg = np.cos(kvec[0] * X + kvec[1] * Y + kvec[2] * Z) * sinc
    del X, Y, Z
    dv = amp * (r[1] * khat + r[2] * t1 + r[3] * t2)
    dp = amp * r[4]
    if mhd:
        db = amp * (r[5] * t1 + r[6] * t2)
        avec = -np.cross(kvec, db) / float(kvec @ kvec)

        def A(x1, x2, x3):
            sn = np.sin(kvec[0] * x1 + kvec[1] * x2 + kvec[2] * x3)
            return (avec[0] * sn, avec[1] * sn, avec[2] * sn)

        b1, b2, b3 = face_field_from_potential(b, A, B0, gl=gl)
        eb = 0.5 * ((0.5 * (b1[:, :, 1:] + b1[:, :, :-1])) ** 2 +
                    (0.5 * (b2[:, 1:, :] + b2[:, :-1, :])) ** 2 +
                    (0.5 * (b3[1:, :, :] + b3[:-1, :, :])) ** 2)
    else:
        nz, ny, nx = shape[2], shape[1], shape[0]
        b1 = np.zeros((nz, ny, nx + 1)); b2 = np.zeros((nz, ny + 1, nx)); b3 = np.zeros((nz + 1, ny, nx))
        eb = 0.0
    cons = np.empty((5,) + cavg.shape)
    cons[0] = 1.0 + amp * r[0] * cavg
    for d in range(3):
        cons[1 + d] = dv[d] * cavg
    cons[4] = (p0 + dp * cavg) / (gamma - 1.0) + eb
    period = (1.0 / float(np.linalg.norm(kvec / (2 * math.pi)))) / lam
    return InitialState(b, cons, b1, b2, b3, gamma,
                        {"speed": lam, "period": period, "amp": amp, "B0": B0})


# ---------------------------------------------------------------------------
# random smooth periodic fields
# ---------------------------------------------------------------------------

def _random_modes(rng, kmax, nmodes):
    ks = rng.integers(-kmax, kmax + 1, size=(nmodes, 3))
    ks[np.all(ks == 0, axis=1)] = (1, 0, 0)
    ph = rng.uniform(0, 2 * math.pi, size=nmodes)
    amp = rng.normal(size=nmodes)
    return ks, ph, amp


def _eval_modes(modes, s1, s2, s3):
    ks, ph, amp = modes
    out = np.zeros(np.broadcast(s1, s2, s3).shape)
    for kv, p, a in zip(ks, ph, amp):
        out = out + a * np.cos(2 * math.pi * (kv[0] * s1 + kv[1] * s2 + kv[2] * s3) + p)
    return out


def smooth_random_mhd(block: Block, seed: int, gamma=5.0 / 3.0, kmax=2, nmodes=6,
                      v_rms=0.5, b_rms=0.5, B0=(0.0, 0.0, 0.0), mhd=True, gl=6) -> InitialState:
    """Random smooth state: rho in [0.5, 2], P in [0.1, 1], v and B from
    low-k random fields (B from a vector potential).  Modes are periodic in
    the block's normalised coordinates s = (x - lo)/(hi - lo)."""
    rng = np.random.default_rng(seed)
    b = block
    X, Y, Z = _cell_mesh(b)
    nrm = lambda x, d: (x - b.lo[d]) / (b.hi[d] - b.lo[d])
    S1, S2, S3 = nrm(X, 0), nrm(Y, 1), nrm(Z, 2)

    def unit(f):
        lo, hi = f.min(), f.max()
        return (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)

    s_rho = unit(_eval_modes(_random_modes(rng, kmax, nmodes), S1, S2, S3))
    s_p = unit(_eval_modes(_random_modes(rng, kmax, nmodes), S1, S2, S3))
    rho = 2.0 ** (2 * s_rho - 1)
    p = 0.1 * 10.0 ** s_p
    v = [_eval_modes(_random_modes(rng, kmax, nmodes), S1, S2, S3) for _ in range(3)]
    vr = math.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)) or 1.0
    v = [q * (v_rms / vr) for q in v]
    if mhd:
        amods = [_random_modes(rng, kmax, nmodes) for _ in range(3)]

        def A(x1, x2, x3):
            t1, t2, t3 = nrm(x1, 0), nrm(x2, 1), nrm(x3, 2)
            return tuple(_eval_modes(m, t1, t2, t3) for m in amods)

        b1, b2, b3 = face_field_from_potential(b, A, (0.0, 0.0, 0.0), gl)
        bc2 = np.mean((0.5 * (b1[:, :, 1:] + b1[:, :, :-1])) ** 2 +
                      (0.5 * (b2[:, 1:, :] + b2[:, :-1, :])) ** 2 +
                      (0.5 * (b3[1:, :, :] + b3[:-1, :, :])) ** 2)
        sc = b_rms / math.sqrt(bc2) if bc2 > 0 else 0.0
        b1, b2, b3 = b1 * sc + B0[0], b2 * sc + B0[1], b3 * sc + B0[2]
    else:
        nx, ny, nz = b.n
        b1, b2, b3 = (np.zeros((nz, ny, nx + 1)), np.zeros((nz, ny + 1, nx)),
                      np.zeros((nz + 1, ny, nx)))
    return _assemble(b, gamma, rho, v, p, b1, b2, b3, {"seed": seed})


# ---------------------------------------------------------------------------
# decaying-turbulence box (256^3 and 512^3 configs)
# ---------------------------------------------------------------------------

def solenoidal_gaussian_velocity(n: int, seed: int, kmin=2.0, kmax=8.0, slope=-2.0):
    """Gaussian random solenoidal field on an n^3 periodic unit cube whose
    shell spectrum E(k) follows k^slope for kmin <= |k| <= kmax (k in units
    of 2 pi / L), normalised to unit rms speed.  Arrays are [z][y][x]."""
    rng = np.random.default_rng(seed)
    kz = np.fft.fftfreq(n, d=1.0 / n)[:, None, None]
    ky = np.fft.fftfreq(n, d=1.0 / n)[None, :, None]
    kx = np.fft.rfftfreq(n, d=1.0 / n)[None, None, :]
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    band = (kk >= kmin) & (kk <= kmax)
    # |v_hat|^2 ~ E(k) / k^2 gives the shell spectrum k^slope
    amp = np.where(band, np.where(kk > 0, kk, 1.0) ** ((slope - 2.0) / 2.0), 0.0)
    comps = []
    for _ in range(3):
        c = rng.normal(size=kk.shape) + 1j * rng.normal(size=kk.shape)
        comps.append(c * amp)
    k2 = np.where(kk > 0, kk ** 2, 1.0)
    kd = (comps[0] * kx + comps[1] * ky + comps[2] * kz) / k2
    comps = [comps[0] - kd * kx, comps[1] - kd * ky, comps[2] - kd * kz]
    v = [np.fft.irfftn(c, s=(n, n, n), axes=(0, 1, 2)) for c in comps]
    rms = math.sqrt(float(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)))
    return [np.ascontiguousarray(q / rms) for q in v]


def turbulence_box(n=256, seed=20260816, mach=2.0, beta=1.0, gamma=1.0001,
                   beta_modulated=False, log_beta=(-1.0, 1.0)) -> InitialState:
    """Decaying MHD turbulence: rho = 1, P = 1/gamma (c_s = 1), uniform B_x
    with plasma beta (or, when beta_modulated, beta varying with y as
    log10 beta = m + a sin(2 pi y) spanning log_beta = (m - a, m + a), by
    default 0.1 .. 10), solenoidal Gaussian velocity, rms Mach `mach`."""
    b = Block((n, n, n))
    v = solenoidal_gaussian_velocity(n, seed)
    v = [q * mach for q in v]
    p0 = 1.0 / gamma
    rho = np.ones((n, n, n))
    p = np.full((n, n, n), p0)
    nx = ny = nz = n
    if beta_modulated:
        yc = b.centers(1)
        m, a = 0.5 * (log_beta[0] + log_beta[1]), 0.5 * (log_beta[1] - log_beta[0])
        bx_row = np.sqrt(2 * p0 / 10.0 ** (m + a * np.sin(2 * math.pi * yc)))   # y only
        b1 = np.broadcast_to(bx_row[None, :, None], (nz, ny, nx + 1)).copy()
    else:
        b1 = np.full((nz, ny, nx + 1), math.sqrt(2 * p0 / beta))
    b2 = np.zeros((nz, ny + 1, nx))
    b3 = np.zeros((nz + 1, ny, nx))
    return _assemble(b, gamma, rho, v, p, b1, b2, b3, {"seed": seed, "mach": mach})


# ---------------------------------------------------------------------------
# 1-D Riemann problems embedded in 3-D
# ---------------------------------------------------------------------------

def taylor_green(n: int, mach: float, gamma=5.0 / 3.0, v0=1.0) -> InitialState:
    """Taylor-Green vortex (the low-Mach dissipation test of Sec. 5): periodic
    [0, 2 pi]^3, rho = 1, v = v0 (sin x cos y cos z, -cos x sin y cos z, 0),
    p = p0 + (v0^2 / 16)(cos 2x + cos 2y)(cos 2z + 2) with p0 = v0^2 /
    (gamma mach^2), so that v0 / c_s = mach; B = 0.  Cell-centre values."""
    b = Block((n, n, n), (0.0, 0.0, 0.0), (2 * math.pi,) * 3)
    X, Y, Z = _cell_mesh(b)
    rho = np.ones_like(X)
    v = (v0 * np.sin(X) * np.cos(Y) * np.cos(Z), -v0 * np.cos(X) * np.sin(Y) * np.cos(Z),
         np.zeros_like(X))
    p0 = v0 * v0 / (gamma * mach * mach)
    p = p0 + (v0 * v0 / 16.0) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    z1 = np.zeros((n, n, n + 1)); z2 = np.zeros((n, n + 1, n)); z3 = np.zeros((n + 1, n, n))
    return _assemble(b, gamma, rho, v, p, z1, z2, z3, {"mach": mach})


def riemann_1d(axis: int, n: int, left: dict, right: dict, gamma: float, x0=0.0,
               lo=-0.5, hi=0.5, ntrans=1) -> InitialState:
    """Discontinuity at x_axis = x0 between primitive states `left` and
    `right` (keys rho, v (3-vector, grid frame), p, B (3-vector)).  Outflow
    along `axis`, periodic (with `ntrans` cells) across it."""
    nn = [ntrans] * 3
    nn[axis] = n
    lo3 = [0.0] * 3
    hi3 = [1.0] * 3
    lo3[axis], hi3[axis] = lo, hi
    bc = [PERIODIC] * 3
    bc[axis] = OUTFLOW
    b = Block(tuple(nn), tuple(lo3), tuple(hi3), CART, tuple(bc))
    X, Y, Z = _cell_mesh(b)
    coord = (X, Y, Z)[axis]
    L = coord < x0
    shape = X.shape
    rho = np.where(L, left["rho"], right["rho"]) * np.ones(shape)
    p = np.where(L, left["p"], right["p"]) * np.ones(shape)
    v = [np.where(L, left["v"][d], right["v"][d]) * np.ones(shape) for d in range(3)]
    nx, ny, nz = b.n
    b1 = np.zeros((nz, ny, nx + 1)); b2 = np.zeros((nz, ny + 1, nx)); b3 = np.zeros((nz + 1, ny, nx))
    fa = [b1, b2, b3]
    for d in range(3):
        bl, br = left.get("B", (0, 0, 0))[d], right.get("B", (0, 0, 0))[d]
        if d == axis:
            # normal component must be uniform for a 1-D problem
            fa[d][...] = bl
        else:
            cc = (X, Y, Z)[axis]
            if d == 0:
                cpos = cc
            elif d == 1:
                cpos = cc
            else:
                cpos = cc
            # tangential faces sit at cell positions along `axis`
            val = np.where(cpos < x0, bl, br)
            if d == 0:
                fa[d][:, :, :-1] = val
                fa[d][:, :, -1] = val[:, :, 0]
            elif d == 1:
                fa[d][:, :-1, :] = val
                fa[d][:, -1, :] = val[:, 0, :]
            else:
                fa[d][:-1, :, :] = val
                fa[d][-1, :, :] = val[0, :, :]
    return _assemble(b, gamma, rho, v, p, b1, b2, b3, {"axis": axis})


SOD_LEFT = {"rho": 1.0, "v": (0.0, 0.0, 0.0), "p": 1.0}
SOD_RIGHT = {"rho": 0.125, "v": (0.0, 0.0, 0.0), "p": 0.1}


def brio_wu(axis: int, n: int) -> InitialState:
    """Brio & Wu (1988) shock tube: gamma = 2, B_n = 0.75, transverse field
    reversing from +1 to -1; the transverse component is the cyclic next
    axis so the problem maps onto itself under axis permutation."""
    t = (axis + 1) % 3
    bl = [0.0, 0.0, 0.0]; br = [0.0, 0.0, 0.0]
    bl[axis] = br[axis] = 0.75
    bl[t], br[t] = 1.0, -1.0
    left = {"rho": 1.0, "v": (0, 0, 0), "p": 1.0, "B": bl}
    right = {"rho": 0.125, "v": (0, 0, 0), "p": 0.1, "B": br}
    return riemann_1d(axis, n, left, right, 2.0)


# ---------------------------------------------------------------------------
# multifluid dust box (128^3 configuration and its smaller parity cases)
# ---------------------------------------------------------------------------

def dust_stopping_times(nd=8, lo=1e-4, hi=1.0):
    """Stopping times log-spaced from lo to hi (units of L / c_s = 1)."""
    return list(np.logspace(math.log10(lo), math.log10(hi), nd))


def dust_box(block: Block, seed: int, nd=8, gamma=5.0 / 3.0, v_rms=0.5, dv_rms=0.1,
             t_stop=None, eps_range=(-3.0, 0.0)):
    """Hydro gas rho = 1, P = 1/gamma (c_s = 1), low-k random velocity of rms
    v_rms; nd pressureless species with dust-to-gas ratios 10^U(eps_range)
    and velocities v_g + dv_k (independent low-k fields of rms dv_rms).
    Returns (gas InitialState, dust[nd][4][nz][ny][nx], t_stop)."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _cell_mesh(block)
    nrm = lambda x, d: (x - block.lo[d]) / (block.hi[d] - block.lo[d])
    S = (nrm(X, 0), nrm(Y, 1), nrm(Z, 2))

    def field(rms):
        comp = [_eval_modes(_random_modes(rng, 2, 6), *S) for _ in range(3)]
        r = math.sqrt(float(np.mean(comp[0] ** 2 + comp[1] ** 2 + comp[2] ** 2))) or 1.0
        return [q * (rms / r) for q in comp]

    vg = field(v_rms)
    shape = X.shape
    rho = np.ones(shape)
    p = np.full(shape, 1.0 / gamma)
    nx, ny, nz = block.n
    z = (np.zeros((nz, ny, nx + 1)), np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx)))
    gas = _assemble(block, gamma, rho, vg, p, *z, {"seed": seed})
    eps = 10.0 ** rng.uniform(eps_range[0], eps_range[1], size=nd)
    dust = np.zeros((nd, 4) + shape)
    for k in range(nd):
        dv = field(dv_rms)
        dust[k, 0] = eps[k] * rho
        for q in range(3):
            dust[k, 1 + q] = dust[k, 0] * (vg[q] + dv[q])
    ts = list(t_stop) if t_stop is not None else dust_stopping_times(nd)
    return gas, np.ascontiguousarray(dust), ts


# ---------------------------------------------------------------------------
# batched independent boxes of uneven sizes (512-box configuration)
# ---------------------------------------------------------------------------

SPH_BOX = dict(lo=(1.0, math.pi / 4, 0.0), hi=(2.0, 3 * math.pi / 4, math.pi / 2))


def _one_box(args):
    b, seed, sizes, sph_every, gamma, nmodes, gl = args
    rng = np.random.default_rng([seed, b])
    n = tuple(int(x) for x in rng.choice(sizes, size=3))
    if sph_every and b % sph_every == sph_every - 1:
        blk = Block(n, SPH_BOX["lo"], SPH_BOX["hi"], SPH, (OUTFLOW, OUTFLOW, PERIODIC))
    else:
        blk = Block(n)
    return smooth_random_mhd(blk, seed + 1 + b, gamma=gamma, nmodes=nmodes, v_rms=0.5,
                             b_rms=0.5, gl=gl)


def batched_boxes(nblocks: int, seed: int, sizes=(16, 24, 32, 48, 64), sph_every=3,
                  gamma=5.0 / 3.0, nmodes=4, gl=6, workers=0):
    """Independent MHD boxes: side lengths drawn uniformly from `sizes` per
    axis; every `sph_every`-th box (block_id % sph_every == sph_every - 1) is
    a spherical-polar wedge r in [1,2], theta in [pi/4, 3pi/4], phi in
    [0, pi/2] (outflow in r and theta, periodic in phi), the others are
    periodic unit boxes.  Fields: random smooth rho in [0.5, 2], P in
    [0.1, 1], low-k v and B (B from a vector potential), rms 0.5."""
    jobs = [(b, seed, tuple(sizes), sph_every, gamma, nmodes, gl) for b in range(nblocks)]
    if workers and workers > 1:
        # spawned workers: safe to use before or after CUDA initialisation
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_one_box, jobs, chunksize=4))
    return [_one_box(j) for j in jobs]


# ---------------------------------------------------------------------------
# learned-flux network: seeded initial parameters
# ---------------------------------------------------------------------------

MLP_DIMS = (14, 128, 128, 128, 7)


def mlp_init_params(seed: int, dims=MLP_DIMS, bias_scale=0.0):
    """Layer-wise N(0, 1/fan_in) weights and (optionally small) biases,
    packed per layer as W[out][in] then b[out] (FP32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(dims) - 1):
        nin, nout = dims[l], dims[l + 1]
        parts.append(rng.normal(size=(nout, nin)) / math.sqrt(nin))
        parts.append(rng.normal(size=nout) * bias_scale)
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def face_states(n: int, seed: int, mhd=True, gamma=5.0 / 3.0, mach=2.0,
                log_beta=(-1.0, 1.0), jumps=((0.70, 1e-3, 2e-2), (0.25, 2e-2, 0.3),
                                              (0.05, 0.3, 1.5))):
    """Random face-frame interface states (wl, wr [n][7], bn [n]; w = rho,
    vn, vt1, vt2, p, Bt1, Bt2) like those of the turbulence workloads: the
    left state has rho log-uniform in [0.3, 3], p = rho^gamma / gamma x
    U(0.5, 2), velocity components N(0, mach / sqrt 3) in units of c_s = 1,
    and (MHD) a field of random direction whose magnitude gives plasma beta
    10^U(log_beta); the right state is the left one with every entry
    perturbed by a relative jump whose size is log-uniform in one of the
    `jumps` classes (fraction, smallest, largest): mostly smooth flow, some
    strong gradients, a few shock-like jumps.  Density and pressure stay
    positive; bn is shared by both sides."""
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(np.log(0.3), np.log(3.0), n))
    p = rho ** gamma / gamma * rng.uniform(0.5, 2.0, n)
    v = rng.normal(size=(n, 3)) * mach / math.sqrt(3.0)
    wl = np.zeros((n, 7))
    wl[:, 0], wl[:, 1:4], wl[:, 4] = rho, v, p
    bn = np.zeros(n)
    if mhd:
        beta = 10.0 ** rng.uniform(log_beta[0], log_beta[1], n)
        bmag = np.sqrt(2.0 * p / beta)
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        bn = bmag * d[:, 0]
        wl[:, 5:7] = bmag[:, None] * d[:, 1:3]
    frac = np.array([j[0] for j in jumps])
    cls = rng.choice(len(jumps), size=n, p=frac / frac.sum())
    lo = np.array([j[1] for j in jumps])[cls]
    hi = np.array([j[2] for j in jumps])[cls]
    size = np.exp(rng.uniform(np.log(lo), np.log(hi)))
    # scale of each entry: the density and pressure themselves, the sound
    # speed for velocities, the field magnitude for fields
    cs = np.sqrt(gamma * p / rho)
    bscale = np.sqrt(bn ** 2 + wl[:, 5] ** 2 + wl[:, 6] ** 2) + 1e-300
    scale = np.stack([rho, cs, cs, cs, p, bscale, bscale], axis=1)
    wr = wl + size[:, None] * scale * rng.normal(size=(n, 7))
    wr[:, 0] = np.maximum(wr[:, 0], 0.2 * wl[:, 0])
    wr[:, 4] = np.maximum(wr[:, 4], 0.2 * wl[:, 4])
    if not mhd:
        wr[:, 5:7] = 0.0
    return wl, wr, bn
