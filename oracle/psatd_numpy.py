"""Second FP64 implementation of the PSATD Maxwell push, in numpy with
scipy.fft as its FFT: a cross-check of the C++ oracle (oracle/psatd_oracle.cpp,
loaded through oracle/psatd_oracle.py), written independently of it.

TEST INFRASTRUCTURE.  Only the CPU tests import this module (they run every
pin against both implementations and compare the two).  The product path
(the CUDA library and its Python binding) never imports it, and this module
imports nothing from the product package.

What it computes (one step = advance every box, then exchange guards; paper
Fig. 1 caption, steps (i) and (ii)):

1. per box, a 3D FFT of every field component over the whole padded box
   (guards included), the box being treated as periodic (Sec. 1.3: local
   shared-memory FFTs on sub-domains padded with n_g guard cells);
2. the per-mode analytical update of Maxwell's equations in Fourier space
   (Sec. 1.1: PSATD, exact in time for every mode), with the derivative
   replaced by the Fourier symbol of an order-p staggered finite-difference
   stencil of width p/2 (Sec. 1.1; p -> infinity gives the pure spectral
   operator) and Yee-staggered field positions;
3. the inverse 3D FFT;
4. the guard exchange: every guard cell receives the value of the interior
   cell that owns the same global position (Fig. 1a/1b, step (ii)).

The paper states the principle of PSATD but prints none of its equations
(they are in its references).  The update used here is derived directly from
Maxwell's equations with the current J held constant over the step:

    dE/dt = c^2 (i K x B) - J/eps0,     dB/dt = -(i K x E),

whose exact solution over dt, with K = |K|, theta = c K dt, C = cos(theta),

    Sw = sin(theta)/(c K)         = dt * sinc(theta)
    X1 = (1 - C)/K^2              = (c dt)^2/2 * sinc(theta/2)^2
    X3 = (Sw - dt)/K^2            = c^2 dt^3 (sinc(theta) - 1)/theta^2

is ("J form"):

    E' = C E + X1 K (K.E) + i c^2 Sw K x B - Sw J/eps0 + X3 K (K.J)/eps0
    B' = C B + X1 K (K.B) - i Sw K x E + i (X1/c^2) K x J/eps0

The X1 K(K.E), X1 K(K.B) terms carry the longitudinal parts (E_L moves only
with J_L, B_L is constant).  With charge density (the "rho form") rho is
advanced by continuity, rho' = rho - i dt K.J, and E takes its longitudinal
part from Gauss's law at the new time:

    E' = C E + i c^2 Sw K x B - Sw J/eps0 + i K (Y1 rho' + Y2 rho)/eps0,
    Y1 = X3/dt,  Y2 = -X1 - X3/dt.

Both forms agree whenever Gauss's law holds at the start of the step.

Fourier convention: forward transform unnormalised with exp(-2 pi i m j/N),
inverse with 1/N; the derivative becomes +i K.  Index m of an axis of N
cells maps to k = 2 pi m~/(N h) with m~ = m for m <= N/2, m - N otherwise
(so the Nyquist index takes k = +pi/h).  A component sampled at offset s
(in cells) is brought to the "centred" spectrum by exp(-i k.s h) before the
update and back by exp(+i k.s h) afterwards.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
from scipy import fft as _fft

# Yee offsets (cells) of every component: E and J on edges, B on faces,
# rho on nodes.
YEE = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Bx": (0.0, 0.5, 0.5), "By": (0.5, 0.0, 0.5), "Bz": (0.5, 0.5, 0.0),
    "Jx": (0.5, 0.0, 0.0), "Jy": (0.0, 0.5, 0.0), "Jz": (0.0, 0.0, 0.5),
    "rho": (0.0, 0.0, 0.0),
}

_WORKERS = int(os.environ.get("PSATD_ORACLE_THREADS", "0")) or (os.cpu_count() or 1)


def fft3(a):
    """Unnormalised forward 3D DFT (library FFT as one step)."""
    return _fft.fftn(a, workers=_WORKERS)


def ifft3(a):
    """Inverse 3D DFT with the 1/N factor."""
    return _fft.ifftn(a, workers=_WORKERS)


# ----------------------------------------------------------------------------
# Order-p staggered stencil (Sec. 1.1: order p, stencil of width p/2)
# ----------------------------------------------------------------------------

def stencil_weights(p: int):
    """Weights alpha_l, l = 1..p/2, of the order-p staggered centred difference

        f'(x) ~ sum_l alpha_l [f(x + (2l-1)h/2) - f(x - (2l-1)h/2)] / ((2l-1) h).

    Exactness to order h^p requires sum_l alpha_l (2l-1)^(2j) = delta_j0 for
    j = 0..p/2-1, whose solution is the Lagrange basis of the nodes (2l-1)^2
    evaluated at 0.  Computed in exact rational arithmetic.  p = 0 (infinite
    order) has no stencil and returns None."""
    if p == 0:
        return None
    if p < 2 or p % 2:
        raise ValueError("order p must be even and >= 2, or 0 for infinite")
    q = p // 2
    nodes = [(2 * l - 1) ** 2 for l in range(1, q + 1)]
    out = []
    for l in range(q):
        a = Fraction(1)
        for j in range(q):
            if j != l:
                a *= Fraction(nodes[j], nodes[j] - nodes[l])
        out.append(a)
    return out


def modified_wavenumber(k, h: float, p: int):
    """Fourier symbol K(k) of the order-p staggered difference (D f = i K f
    in centred form); the pure spectral operator K = k for p = 0."""
    k = np.asarray(k, dtype=np.float64)
    if p == 0:
        return k.copy()
    K = np.zeros_like(k)
    for l, a in enumerate(stencil_weights(p), start=1):
        m = 2 * l - 1
        K += float(a) * 2.0 * np.sin(m * k * h / 2.0) / (m * h)
    return K


def nodal_weights(p: int):
    """Weights beta_l, l = 1..p/2, of the order-p centred difference on a
    collocated (nodal) grid

        f'(x) ~ sum_l beta_l [f(x + l h) - f(x - l h)] / (2 l h),

    exact to order h^p: sum_l beta_l l^(2j) = delta_j0 for j = 0..p/2-1, the
    Lagrange basis of the nodes l^2 evaluated at 0 (exact rationals).  This
    variant (all components at the cell nodes, no Yee shifts) is not in the
    paper, which uses staggered stencils; p = 0 returns None."""
    if p == 0:
        return None
    if p < 2 or p % 2:
        raise ValueError("order p must be even and >= 2, or 0 for infinite")
    q = p // 2
    out = []
    for l in range(1, q + 1):
        b = Fraction(1)
        for j in range(1, q + 1):
            if j != l:
                b *= Fraction(j * j, j * j - l * l)
        out.append(b)
    return out


def modified_wavenumber_nodal(k, h: float, p: int):
    """Fourier symbol K(k) = sum_l beta_l sin(l k h)/(l h) of the order-p
    centred nodal difference (D f = i K f); K = k for p = 0 except at the
    Nyquist wavenumber |k| = pi/h, where K = 0: on a collocated grid the
    Nyquist mode is its own mirror image (k = -k), so only K = 0 keeps the
    derivative of a real field real (finite p gives 0 there by itself)."""
    k = np.asarray(k, dtype=np.float64)
    if p == 0:
        K = k.copy()
        K[np.isclose(np.abs(k * h), np.pi, rtol=0, atol=1e-12)] = 0.0
        return K
    K = np.zeros_like(k)
    for l, b in enumerate(nodal_weights(p), start=1):
        K += float(b) * np.sin(l * k * h) / (l * h)
    return K


def axis_wavenumbers(n: int, h: float):
    """True wavenumber of every index of an n-point periodic axis."""
    m = np.arange(n)
    mt = np.where(m <= n // 2, m, m - n)
    return 2.0 * np.pi * mt / (n * h)


# ----------------------------------------------------------------------------
# Per-mode coefficients and update (Sec. 1.1, PSATD)
# ----------------------------------------------------------------------------

def _sinc(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = np.sin(x[nz]) / x[nz]
    return out


def coefficients(K2, c: float, dt: float):
    """C, Sw, X1, X3 of the module docstring as functions of K^2.

    1 - C is evaluated as 2 sin^2(theta/2) (through sinc(theta/2)) so that it
    keeps full relative precision at small theta; (sinc(theta) - 1)/theta^2
    uses its Taylor series below theta = 0.1, where the difference would
    cancel, and takes the value -1/6 at K = 0."""
    K2 = np.asarray(K2, dtype=np.float64)
    th = c * dt * np.sqrt(K2)
    C = np.cos(th)
    Sw = dt * _sinc(th)
    X1 = 0.5 * (c * dt) ** 2 * _sinc(0.5 * th) ** 2
    t2 = th * th
    small = np.abs(th) < 0.1
    g = np.empty_like(th)
    # (sinc(t) - 1)/t^2 = sum_{j>=1} (-1)^j t^(2j-2)/(2j+1)!
    ts = t2[small]
    g[small] = (-1.0 / 6 + ts * (1.0 / 120 + ts * (-1.0 / 5040 + ts * (1.0 / 362880
               + ts * (-1.0 / 39916800)))))
    big = ~small
    g[big] = (np.sin(th[big]) / th[big] - 1.0) / t2[big]
    X3 = c * c * dt ** 3 * g
    return C, Sw, X1, X3


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1],
            a[2] * b[0] - a[0] * b[2],
            a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def update_modes(E, B, J, R, K, dt, c=1.0, eps0=1.0, form="vacuum"):
    """Advance centred spectra by one step of dt.

    E, B: 3-tuples of complex arrays; J: 3-tuple or None; R: rho array or
    None; K: 3-tuple of real arrays (modified wavenumber components).
    form: 'vacuum' (J = rho = 0), 'J' (J form) or 'rho' (rho form).
    Returns (E', B', rho') with rho' None unless form == 'rho'."""
    K2 = _dot(K, K)
    C, Sw, X1, X3 = coefficients(K2, c, dt)
    KxB = _cross(K, B)
    KxE = _cross(K, E)
    KdB = _dot(K, B)
    Bn = [C * B[d] + X1 * K[d] * KdB - 1j * Sw * KxE[d] for d in range(3)]
    if form == "rho":
        KdJ = _dot(K, J)
        Rn = R - 1j * dt * KdJ
        Y1 = X3 / dt
        Y2 = -X1 - X3 / dt
        En = [C * E[d] + 1j * c * c * Sw * KxB[d] - Sw * J[d] / eps0
              + 1j * K[d] * (Y1 * Rn + Y2 * R) / eps0 for d in range(3)]
    else:
        KdE = _dot(K, E)
        En = [C * E[d] + X1 * K[d] * KdE + 1j * c * c * Sw * KxB[d] for d in range(3)]
        Rn = None
        if form == "J":
            KdJ = _dot(K, J)
            En = [En[d] - Sw * J[d] / eps0 + X3 * K[d] * KdJ / eps0 for d in range(3)]
        elif form != "vacuum":
            raise ValueError(form)
    if form in ("J", "rho"):
        KxJ = _cross(K, J)
        Bn = [Bn[d] + 1j * (X1 / (c * c)) * KxJ[d] / eps0 for d in range(3)]
    return En, Bn, Rn


def _box_k(shape_zyx, h, p, nodal=False):
    """Broadcastable (k, K) grids for a box: true and modified wavenumbers."""
    nz, ny, nx = shape_zyx
    kx = axis_wavenumbers(nx, h[0])[None, None, :]
    ky = axis_wavenumbers(ny, h[1])[None, :, None]
    kz = axis_wavenumbers(nz, h[2])[:, None, None]
    mw = modified_wavenumber_nodal if nodal else modified_wavenumber
    Kx = mw(kx, h[0], p)
    Ky = mw(ky, h[1], p)
    Kz = mw(kz, h[2], p)
    return (kx, ky, kz), (Kx, Ky, Kz)


def _shift(k, comp, h, sign, nodal=False):
    if nodal:                     # every component at the cell nodes
        return 1.0
    s = YEE[comp]
    return np.exp(sign * 1j * (k[0] * s[0] * h[0] + k[1] * s[1] * h[1] + k[2] * s[2] * h[2]))


def push_box(f, src, h, p, dt, c=1.0, eps0=1.0, form="vacuum", return_imag=False, nodal=False):
    """One PSATD step on one periodic box.

    f: dict Ex..Bz -> (nz, ny, nx) float64 arrays; src: dict Jx, Jy, Jz[, rho]
    or None.  Returns a new dict (with 'rho' when form == 'rho').  nodal: the
    collocated variant (nodal_weights, no Yee shifts)."""
    shape = f["Ex"].shape
    k, K = _box_k(shape, h, p, nodal)
    cen = lambda a, comp: fft3(a) * _shift(k, comp, h, -1.0, nodal)
    E = tuple(cen(f[c_], c_) for c_ in ("Ex", "Ey", "Ez"))
    B = tuple(cen(f[c_], c_) for c_ in ("Bx", "By", "Bz"))
    J = R = None
    if form in ("J", "rho"):
        J = tuple(cen(src[c_], c_) for c_ in ("Jx", "Jy", "Jz"))
    if form == "rho":
        R = cen(src["rho"], "rho")
    En, Bn, Rn = update_modes(E, B, J, R, K, dt, c, eps0, form)
    out, imag = {}, 0.0
    for comp, a in zip(("Ex", "Ey", "Ez", "Bx", "By", "Bz"), list(En) + list(Bn)):
        r = ifft3(a * _shift(k, comp, h, +1.0, nodal))
        imag = max(imag, float(np.abs(r.imag).max()))
        out[comp] = r.real.copy()
    if Rn is not None:
        r = ifft3(Rn)
        imag = max(imag, float(np.abs(r.imag).max()))
        out["rho"] = r.real.copy()
    if return_imag:
        return out, imag
    return out


# ----------------------------------------------------------------------------
# Guard exchange (Fig. 1, step (ii); Sec. 2.1 for groups)
# ----------------------------------------------------------------------------

def _interior_slices(box):
    return tuple(slice(box.ng_lo[d], box.n[d] - box.ng_hi[d]) for d in (2, 1, 0))


def _assemble(layout, arrays):
    """The global field from the box interiors (they must tile the domain)."""
    gn = layout.global_n
    G = np.zeros((gn[2], gn[1], gn[0]))
    cover = np.zeros(G.shape, dtype=np.int64)
    for b, a in zip(layout.boxes, arrays):
        o, m = b.origin, b.interior
        dst = (slice(o[2], o[2] + m[2]), slice(o[1], o[1] + m[1]), slice(o[0], o[0] + m[0]))
        G[dst] = a[_interior_slices(b)]
        cover[dst] += 1
    if not (cover == 1).all():
        raise ValueError("box interiors do not tile the global domain")
    return G


def _sample(layout, G):
    """Per-box arrays whose every padded cell reads the global cell at
    origin - ng_lo + i (periodic axes wrap, non-periodic axes give 0 outside
    the domain)."""
    gn = layout.global_n
    Gz = np.zeros((gn[2] + 1, gn[1] + 1, gn[0] + 1))
    Gz[:-1, :-1, :-1] = G                      # index -1 reads the zero plane
    out = []
    for b in layout.boxes:
        idx = []
        for d in range(3):
            g = b.origin[d] - b.ng_lo[d] + np.arange(b.n[d])
            if layout.periodic[d]:
                g = g % gn[d]
            else:
                g = np.where((g >= 0) & (g < gn[d]), g, -1)
            idx.append(g)
        out.append(np.ascontiguousarray(Gz[np.ix_(idx[2], idx[1], idx[0])]))
    return out


def exchange(layout, arrays):
    """Return new per-box arrays whose guards hold the owning interior values.

    Non-independent layouts: the box interiors tile the global domain; the
    global field is assembled from them and every padded cell reads the
    global cell at origin - ng_lo + i (periodic axes wrap, non-periodic axes
    give 0 outside the domain).  Independent boxes wrap onto their own
    interior."""
    if layout.kind == "independent":
        out = []
        for b, a in zip(layout.boxes, arrays):
            inner = a[_interior_slices(b)]
            idx = [(np.arange(b.n[d]) - b.ng_lo[d]) % b.interior[d] for d in range(3)]
            out.append(np.ascontiguousarray(inner[np.ix_(idx[2], idx[1], idx[0])]))
        return out
    return _sample(layout, _assemble(layout, arrays))


def couple(src_layout, src_arrays, dst_layout):
    """Dual-grid coupling (paper Sec. 2.5.2, dual grid decomposition): two
    decompositions of the same global domain; every cell of every destination
    box (guards included) takes the value of the source-layout interior cell
    with the same global index (periodic wrap; 0 outside a non-periodic
    domain).  G1 -> G2 fills the FFT grid, guards included; G2 -> G1 copies
    the FFT grid's interiors back."""
    if tuple(src_layout.global_n) != tuple(dst_layout.global_n) or \
            tuple(src_layout.periodic) != tuple(dst_layout.periodic):
        raise ValueError("layouts of different domains")
    return _sample(dst_layout, _assemble(src_layout, src_arrays))


# ----------------------------------------------------------------------------
# Whole push over a layout
# ----------------------------------------------------------------------------

COMPS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


def push(layout, fields, src, nsteps, h, dt, c=1.0, eps0=1.0, form="vacuum",
         boxes=None, nodal=False):
    """Advance ``fields`` (dict comp -> list of per-box arrays) by ``nsteps``
    steps: every step advances each box (Sec. 1.3 local FFT), then exchanges
    guards.  With form 'rho', ``src['rho']`` is advanced too and returned in
    the output dict.  ``boxes`` restricts the advance to a subset (no
    exchange then), for sampled checks of large layouts."""
    cur = {k: list(v) for k, v in fields.items()}
    rho = list(src["rho"]) if form == "rho" else None
    sel = range(len(layout.boxes)) if boxes is None else boxes
    for _ in range(nsteps):
        new = {k: list(v) for k, v in cur.items()}
        new_rho = list(rho) if rho is not None else None
        for b in sel:
            box = layout.boxes[b]
            fb = {k: cur[k][b] for k in COMPS}
            sb = None
            if form in ("J", "rho"):
                sb = {k: src[k][b] for k in ("Jx", "Jy", "Jz")}
                if form == "rho":
                    sb["rho"] = rho[b]
            o = push_box(fb, sb, h, box.p, dt, c, eps0, form, nodal=nodal)
            for k in COMPS:
                new[k][b] = o[k]
            if form == "rho":
                new_rho[b] = o["rho"]
        has_guards = any(g for b in layout.boxes for g in b.ng_lo + b.ng_hi)
        if boxes is None and has_guards:
            for k in COMPS:
                new[k] = exchange(layout, new[k])
            if new_rho is not None:
                new_rho = exchange(layout, new_rho)
        cur, rho = new, new_rho
    if rho is not None:
        cur["rho"] = rho
    return cur


# ----------------------------------------------------------------------------
# Memory model of the decompositions (Sec. 2.2, eqs. (1)-(6); Sec. 2.3, eq. (7))
# ----------------------------------------------------------------------------

def memory_local(n, n_p, n_g):
    """Eq. (1): field cells of the local solver, n_p^3 (n/n_p + 2 n_g)^3."""
    return n_p ** 3 * (n / n_p + 2 * n_g) ** 3


def memory_hybrid(n, n_p, n_g, n_mpi):
    """Eq. (3): (n_p/n_mpi)^3 (n n_mpi/n_p + 2 n_g)^3."""
    return (n_p / n_mpi) ** 3 * (n * n_mpi / n_p + 2 * n_g) ** 3


def memory_gain(d, n_mpi):
    """Eq. (6): G^d = 3^d (n_mpi/(2 + n_mpi))^d at n/n_p = n_g."""
    return 3 ** d * (n_mpi / (2.0 + n_mpi)) ** d


def guard_gain(d, n_mpi):
    """Eq. (7): (3^d - 1)/((1 + 2/n_mpi)^d - 1)."""
    return (3 ** d - 1) / ((1 + 2.0 / n_mpi) ** d - 1)


# ----------------------------------------------------------------------------
# Error metrics (relative L2 and max norm over interior cells)
# ----------------------------------------------------------------------------

def interior(layout, arrays):
    return [a[_interior_slices(b)] for b, a in zip(layout.boxes, arrays)]


def rel_errors(layout, got, ref):
    """Relative L2 and max-norm error of per-box arrays over interior cells;
    absolute when the reference is identically zero."""
    g = np.concatenate([x.ravel() for x in interior(layout, got)])
    r = np.concatenate([x.ravel() for x in interior(layout, ref)])
    d = g - r
    nr = np.linalg.norm(r)
    mr = np.abs(r).max() if r.size else 0.0
    l2 = np.linalg.norm(d) / nr if nr > 0 else np.linalg.norm(d)
    mx = np.abs(d).max() / mr if mr > 0 else (np.abs(d).max() if d.size else 0.0)
    return float(l2), float(mx)


def rel_l2_fields(layout, got, ref, comps):
    """Relative L2 over a vector field (all listed components together)."""
    num = den = 0.0
    for k in comps:
        for b, a, r in zip(layout.boxes, got[k], ref[k]):
            s = _interior_slices(b)
            num += float(np.sum((a[s] - r[s]) ** 2))
            den += float(np.sum(r[s] ** 2))
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)
