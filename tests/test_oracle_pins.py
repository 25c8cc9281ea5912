"""Pins of the FP64 oracle to facts fixed outside it (CPU only).

Each check uses an independent route: a brute-force DFT, exact rational
arithmetic, real-space finite-difference stencils applied cell by cell, the
matrix exponential of the Maxwell generator, analytic plane waves, invariants
of Maxwell's equations, and the values the paper prints for its memory model.

Every pin runs against both implementations: the oracle (C++ with its own
FFT, oracle/psatd_oracle.cpp) and the numpy/scipy cross-check
(oracle/psatd_numpy.py).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from oracle import psatd_numpy, psatd_oracle
from paper_1812_07357_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
IMPLS = {"cpp": psatd_oracle, "numpy": psatd_numpy}


@pytest.fixture(params=sorted(IMPLS))
def O(request):
    """The implementation under test."""
    return IMPLS[request.param]


# ---------------------------------------------------------------------------
# test-side helpers (independent of the oracle's Fourier-space formulas)
# ---------------------------------------------------------------------------

def direct_dft_1d(x):
    n = len(x)
    j = np.arange(n)
    return np.array([np.sum(x * np.exp(-2j * np.pi * m * j / n)) for m in range(n)])


def vandermonde_weights(p):
    """Solve sum_l w_l (2l-1)^(2j) = delta_j0 (j < p/2) by Gaussian elimination
    over the rationals."""
    q = p // 2
    A = [[Fraction((2 * l - 1) ** (2 * j)) for l in range(1, q + 1)] + [Fraction(int(j == 0))]
         for j in range(q)]
    for c in range(q):
        piv = next(r for r in range(c, q) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        for r in range(q):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [A[r][q] / A[r][r] for r in range(q)]


def stag_diff(f, axis, p, h, from_half):
    """Order-p staggered difference along ``axis`` (numpy axis) of a periodic
    array.  from_half=False: samples at integer nodes -> result at j+1/2;
    from_half=True: samples at j+1/2 -> result at integer nodes."""
    w = vandermonde_weights(p)
    out = np.zeros_like(f)
    for l, a in enumerate(w, start=1):
        m = 2 * l - 1
        if from_half:
            plus, minus = np.roll(f, -(l - 1), axis), np.roll(f, l, axis)
        else:
            plus, minus = np.roll(f, -l, axis), np.roll(f, l - 1, axis)
        out += float(a) * (plus - minus) / (m * h)
    return out


AX = {"x": 2, "y": 1, "z": 0}


def D(f, comp, d, p, h=1.0):
    """Derivative along axis d ('x','y','z') of component ``comp`` (Yee)."""
    s = psatd_oracle.YEE[comp]["xyz".index(d)]
    return stag_diff(f, AX[d], p, h, from_half=(s == 0.5))


def div_B(f, p):
    return D(f["Bx"], "Bx", "x", p) + D(f["By"], "By", "y", p) + D(f["Bz"], "Bz", "z", p)


def div_E(f, p):
    return D(f["Ex"], "Ex", "x", p) + D(f["Ey"], "Ey", "y", p) + D(f["Ez"], "Ez", "z", p)


def energy(f):
    return sum(float(np.sum(f[k] ** 2)) for k in psatd_oracle.COMPS)


def one_box(layout, d):
    return {k: [v] for k, v in d.items()}


# ---------------------------------------------------------------------------
# FFT
# ---------------------------------------------------------------------------

def _five_smooth(n):
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


@pytest.mark.parametrize("n", [n for n in range(2, 65, 2) if _five_smooth(n)])
def test_fft_1d_matches_direct_dft(O, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = O.fft3(x.reshape(1, 1, n)).ravel()
    ref = direct_dft_1d(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(4, 6, 10), (6, 4, 8), (10, 12, 6)])
def test_fft_3d_matches_direct_dft(O, shape):
    rng = np.random.default_rng(1)
    a = rng.standard_normal(shape)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ref = np.empty(shape, complex)
    for mz in range(nz):
        for my in range(ny):
            for mx in range(nx):
                ph = np.exp(-2j * np.pi * (mx * x / nx + my * y / ny + mz * z / nz))
                ref[mz, my, mx] = np.sum(a * ph)
    got = O.fft3(a)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    back = O.ifft3(got)
    assert np.max(np.abs(back - a)) <= 1e-13


# ---------------------------------------------------------------------------
# Stencil weights and modified wavenumber (Sec. 1.1: order p, width p/2)
# ---------------------------------------------------------------------------

def _same(w, exact, rel=4e-15):
    """w (exact rationals, or floats of the C++ oracle) against exact values:
    equal for rationals, within `rel` relative for floats."""
    assert len(w) == len(exact)
    for a, e in zip(w, exact):
        if isinstance(a, Fraction):
            assert a == e
        else:
            assert abs(Fraction(a) - e) <= rel * abs(e), (a, e)


def _exactness(w, nodes_pow, p):
    """sum_l w_l node_l^(2j) = delta_j0 for j < p/2: exact for rationals; for
    floats within 1e-13 of the magnitude of the terms (summed exactly)."""
    for j in range(p // 2):
        terms = [Fraction(a) * nodes_pow(l) ** (2 * j) for l, a in enumerate(w, start=1)]
        s = sum(terms)
        want = 1 if j == 0 else 0
        if all(isinstance(a, Fraction) for a in w):
            assert s == want
        else:
            assert abs(s - want) <= Fraction(1, 10 ** 13) * sum(abs(t) for t in terms), (p, j)


def test_stencil_weights_low_orders(O):
    _same(O.stencil_weights(2), [Fraction(1)])
    _same(O.stencil_weights(4), [Fraction(9, 8), Fraction(-1, 8)])
    # the classical 4th-order staggered coefficients 9/8 and -1/24
    w = O.stencil_weights(4)
    _same([w[0] / 1, w[1] / 3], [Fraction(9, 8), Fraction(-1, 24)])
    assert O.stencil_weights(0) is None


@pytest.mark.parametrize("p", [2, 4, 6, 8, 16, 32, 64])
def test_stencil_weights_exactness(O, p):
    w = O.stencil_weights(p)
    assert len(w) == p // 2            # stencil of width p/2 per side
    _exactness(w, lambda l: 2 * l - 1, p)
    if p <= 16:
        _same(w, vandermonde_weights(p), rel=1e-14)


@pytest.mark.parametrize("p", [2, 4, 8, 16])
def test_modified_wavenumber_is_stencil_eigenvalue(O, p):
    n, h = 24, 0.7
    x = np.arange(n)
    for m in range(0, n // 2 + 1):
        k = 2 * np.pi * m / (n * h)
        f = np.exp(1j * k * x * h).reshape(1, 1, n)   # samples at integer nodes
        g = stag_diff(f, 2, p, h, from_half=False).ravel()  # at j + 1/2
        # centred symbol: g(x_j + h/2) = i K f(x_j + h/2)
        lam = g / np.exp(1j * k * (x + 0.5) * h)
        K = O.modified_wavenumber(k, h, p)
        assert np.allclose(lam, 1j * K, atol=1e-12, rtol=0)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_modified_wavenumber_order(O, p):
    h = 1.0
    e1 = abs(O.modified_wavenumber(0.2, h, p) - 0.2)
    e2 = abs(O.modified_wavenumber(0.1, h, p) - 0.1)
    # error ~ k^(p+1)
    assert 2 ** (p + 1) * 0.8 < e1 / e2 < 2 ** (p + 1) * 1.2
    assert O.modified_wavenumber(0.3, h, 0) == 0.3


def test_modified_wavenumber_monotone(O):
    # K strictly increasing on (0, pi/h]: K = 0 only at k = 0.
    k = np.linspace(1e-6, np.pi, 2000)
    for p in (2, 4, 8, 16, 32, 64):
        K = O.modified_wavenumber(k, 1.0, p)
        assert np.all(np.diff(K) > 0) and K[0] > 0


# ---------------------------------------------------------------------------
# Per-mode update = exact solution of the mode's Maxwell ODE (Sec. 1.1)
# ---------------------------------------------------------------------------

def _generator(K, c, eps0):
    """12x12 generator of d/dt [E, B, J] = [c^2 iKxB - J/eps0, -iKxE, 0]
    extended with rho: d rho/dt = -i K.J (13x13)."""
    def cross_mat(k):
        return np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]], complex)
    X = cross_mat(K)
    A = np.zeros((13, 13), complex)
    A[0:3, 3:6] = 1j * c * c * X
    A[0:3, 6:9] = -np.eye(3) / eps0
    A[3:6, 0:3] = -1j * X
    A[12, 6:9] = -1j * np.asarray(K)
    return A


@pytest.mark.parametrize("form", ["vacuum", "J", "rho"])
def test_update_equals_matrix_exponential(O, form):
    rng = np.random.default_rng(7)
    c, eps0, dt = 1.3, 0.8, 0.9
    Ks = [rng.standard_normal(3) * s for s in (2.0, 1.0, 0.3, 1e-3, 1e-6)]
    Ks.append(np.zeros(3))
    Ks.append(np.array([np.pi, 0.0, 0.0]))
    for K in Ks:
        v = rng.standard_normal(13) + 1j * rng.standard_normal(13)
        if form == "vacuum":
            v[6:9] = 0
        if form == "rho":
            v[12] = 1j * eps0 * np.dot(K, v[0:3])       # Gauss's law at t = 0
        ref = scipy.linalg.expm(dt * _generator(K, c, eps0)) @ v
        E = tuple(np.array([v[d]]) for d in range(3))
        B = tuple(np.array([v[3 + d]]) for d in range(3))
        J = tuple(np.array([v[6 + d]]) for d in range(3))
        R = np.array([v[12]])
        Kt = tuple(np.array([K[d]]) for d in range(3))
        En, Bn, Rn = O.update_modes(E, B, J, R, Kt, dt, c, eps0, form)
        got = np.array([e[0] for e in En] + [b[0] for b in Bn])
        scale = np.max(np.abs(ref[:6])) + 1
        assert np.max(np.abs(got - ref[:6])) <= 1e-12 * scale, (form, K)
        if form == "rho":
            assert abs(Rn[0] - ref[12]) <= 1e-12 * (abs(ref[12]) + 1)


def test_coefficients_small_theta_continuity(O):
    # the Taylor branch and the direct branch meet smoothly at theta = 0.1
    K2 = np.array([(0.1 * (1 - 1e-9)) ** 2, (0.1 * (1 + 1e-9)) ** 2])
    C, Sw, X1, X3 = O.coefficients(K2, 1.0, 1.0)
    assert abs(X3[0] - X3[1]) < 1e-11
    C0, Sw0, X10, X30 = O.coefficients(np.array([0.0]), 2.0, 0.5)
    assert C0[0] == 1.0 and Sw0[0] == 0.5
    assert abs(X10[0] - 0.5 * (2.0 * 0.5) ** 2) < 1e-16
    assert abs(X30[0] - (-(2.0 ** 2) * 0.5 ** 3 / 6)) < 1e-16


# ---------------------------------------------------------------------------
# Whole push: analytic solutions and invariants
# ---------------------------------------------------------------------------

def test_plane_waves_analytic_infinite_order(O):
    """32^3, p = infinity, dt = 0.5, 64 steps: exact to rounding (Sec. 1.1:
    accurate to machine precision, no numerical dispersion)."""
    w = I.make_workload("plane_waves_32")
    out = O.push(w.layout, w.fields, w.src, w.steps, w.h, w.dt, form="vacuum")
    ref = I.plane_wave_fields(I.plane_wave_set(seed=1), (32, 32, 32), w.h, 1.0, w.steps * w.dt)
    refb = {k: [v] for k, v in ref.items()}
    assert O.rel_l2_fields(w.layout, out, refb, O.COMPS) < 1e-12


def test_no_courant_limit_in_vacuum(O):
    """dt = 5 cells at infinite order still matches the analytic waves."""
    n = 16
    lay = I.global_layout((n, n, n), 0)
    waves = I.plane_wave_set(seed=3, mmax=3)
    f0 = {k: [v] for k, v in I.plane_wave_fields(waves, (n, n, n)).items()}
    out = O.push(lay, f0, {}, 3, (1.0,) * 3, 5.0)
    ref = {k: [v] for k, v in I.plane_wave_fields(waves, (n, n, n), t=15.0).items()}
    assert O.rel_l2_fields(lay, out, ref, O.COMPS) < 1e-12


@pytest.mark.parametrize("p", [2, 4, 16])
def test_dispersion_relation_finite_order(O, p):
    """A standing wave E_y = cos(kx) oscillates with omega = c K_p(k), K_p
    the eigenvalue of the real-space stencil."""
    n, h, dt, c = 32, 1.0, 0.3, 1.0
    lay = I.global_layout((n, n, n), p)
    for m in (1, 5, 11, 16):
        k = 2 * np.pi * m / n
        x = np.arange(n)
        f = {key: np.zeros((n, n, n)) for key in O.COMPS}
        f["Ey"][:] = np.cos(k * x * h)[None, None, :]
        out = O.push(lay, one_box(lay, f), {}, 1, (h,) * 3, dt)
        ratio = out["Ey"][0][0, 0, 0] / f["Ey"][0, 0, 0]
        # independent K: apply the stencil to exp(ikx) in real space
        e = np.exp(1j * k * x * h).reshape(1, 1, n)
        lam = (stag_diff(e, 2, p, h, from_half=False).ravel()[3]
               / np.exp(1j * k * (3.5) * h))
        Kp = lam.imag
        assert abs(ratio - math.cos(c * Kp * dt)) < 1e-13


def test_divB_stays_zero_under_stencil_divergence(O):
    rng = np.random.default_rng(11)
    n, p = 12, 8
    lay = I.global_layout((n, n + 4, n - 2), p)
    shp = lay.boxes[0].shape
    A = {k: rng.standard_normal(shp) for k in ("Ex", "Ey", "Ez")}   # A at E positions
    f = {k: rng.standard_normal(shp) for k in ("Ex", "Ey", "Ez")}
    f["Bx"] = D(A["Ez"], "Ez", "y", p) - D(A["Ey"], "Ey", "z", p)
    f["By"] = D(A["Ex"], "Ex", "z", p) - D(A["Ez"], "Ez", "x", p)
    f["Bz"] = D(A["Ey"], "Ey", "x", p) - D(A["Ex"], "Ex", "y", p)
    assert np.abs(div_B(f, p)).max() < 1e-12
    j = {k: rng.standard_normal(shp) for k in ("Jx", "Jy", "Jz")}
    out = O.push(lay, one_box(lay, f), one_box(lay, j), 5, (1.0,) * 3, 0.7, form="J")
    fb = {k: v[0] for k, v in out.items()}
    assert np.abs(div_B(fb, p)).max() < 1e-11 * max(1.0, np.abs(fb["Bx"]).max())


@pytest.mark.parametrize("form", ["rho", "J"])
def test_gauss_law_kept_with_continuity_consistent_current(O, form):
    rng = np.random.default_rng(12)
    n, p, dt = 12, 4, 0.9
    lay = I.global_layout((n, n, n), p)
    shp = lay.boxes[0].shape
    f = {k: np.zeros(shp) for k in O.COMPS}
    j = {k: rng.standard_normal(shp) for k in ("Jx", "Jy", "Jz")}
    j["rho"] = np.zeros(shp)
    nsteps = 4
    out = O.push(lay, one_box(lay, f), one_box(lay, j), nsteps, (1.0,) * 3, dt, form="rho")
    fb = {k: v[0] for k, v in out.items()}
    rho = fb["rho"]
    # continuity, cell by cell: rho_n = -n dt div J
    divJ = div_E({"Ex": j["Jx"], "Ey": j["Jy"], "Ez": j["Jz"]}, p)
    assert np.abs(rho + nsteps * dt * divJ).max() < 1e-11
    assert np.abs(div_E(fb, p) - rho).max() < 1e-11
    if form == "J":
        outj = O.push(lay, one_box(lay, f), one_box(lay, j), nsteps, (1.0,) * 3, dt, form="J")
        for k in O.COMPS:
            assert np.abs(outj[k][0] - fb[k]).max() < 1e-11


def test_vacuum_energy_conserved(O):
    rng = np.random.default_rng(13)
    lay = I.global_layout((10, 12, 8), 16)
    shp = lay.boxes[0].shape
    f = {k: rng.standard_normal(shp) for k in O.COMPS}
    out = O.push(lay, one_box(lay, f), {}, 7, (1.0, 0.8, 1.3), 1.1)
    e0 = energy(f)
    e1 = energy({k: v[0] for k, v in out.items()})
    assert abs(e1 - e0) < 1e-12 * e0


def test_time_reversal(O):
    rng = np.random.default_rng(14)
    lay = I.global_layout((12, 10, 8), 8)
    shp = lay.boxes[0].shape
    f = {k: rng.standard_normal(shp) for k in O.COMPS}
    fw = O.push(lay, one_box(lay, f), {}, 5, (1.0,) * 3, 0.6)
    bw = O.push(lay, fw, {}, 5, (1.0,) * 3, -0.6)
    for k in O.COMPS:
        assert np.abs(bw[k][0] - f[k]).max() < 1e-12


@pytest.mark.parametrize("form", ["vacuum", "J", "rho"])
def test_semigroup(O, form):
    rng = np.random.default_rng(15)
    lay = I.global_layout((8, 10, 12), 16)
    shp = lay.boxes[0].shape
    f = {k: rng.standard_normal(shp) for k in O.COMPS}
    s = {k: rng.standard_normal(shp) for k in ("Jx", "Jy", "Jz")}
    s["rho"] = np.zeros(shp)
    if form == "rho":
        f = {k: np.zeros(shp) for k in O.COMPS}
    a = O.push(lay, one_box(lay, f), one_box(lay, s), 6, (1.0,) * 3, 0.45, form=form)
    b = O.push(lay, one_box(lay, f), one_box(lay, s), 1, (1.0,) * 3, 6 * 0.45, form=form)
    for k in a:
        assert np.abs(a[k][0] - b[k][0]).max() < 1e-11 * (1 + np.abs(b[k][0]).max())


def test_result_is_real(O):
    rng = np.random.default_rng(16)
    f = {k: rng.standard_normal((8, 10, 12)) for k in O.COMPS}
    s = {k: rng.standard_normal((8, 10, 12)) for k in ("Jx", "Jy", "Jz", "rho")}
    for p in (0, 2, 32):
        _, imag = O.push_box(f, s, (1.0, 1.1, 0.9), p, 0.9, form="rho", return_imag=True)
        assert imag < 1e-13


# ---------------------------------------------------------------------------
# Guard exchange (Fig. 1, step (ii)) against a cell-by-cell owner search
# ---------------------------------------------------------------------------

def _brute_exchange(layout, arrays):
    out = []
    for b in layout.boxes:
        a = np.zeros(b.shape)
        for kz in range(b.n[2]):
            for ky in range(b.n[1]):
                for kx in range(b.n[0]):
                    loc = (kx, ky, kz)
                    if layout.kind == "independent":
                        m = b.interior
                        src_b = b
                        gl = tuple((loc[d] - b.ng_lo[d]) % m[d] for d in range(3))
                        src = layout.boxes.index(b)
                        li = tuple(gl[d] + b.ng_lo[d] for d in range(3))
                        a[kz, ky, kx] = arrays[src][li[2], li[1], li[0]]
                        continue
                    g = [b.origin[d] - b.ng_lo[d] + loc[d] for d in range(3)]
                    outside = False
                    for d in range(3):
                        if layout.periodic[d]:
                            g[d] %= layout.global_n[d]
                        elif not 0 <= g[d] < layout.global_n[d]:
                            outside = True
                    if outside:
                        continue
                    hits = []
                    for s, sb in enumerate(layout.boxes):
                        if all(sb.origin[d] <= g[d] < sb.origin[d] + sb.interior[d] for d in range(3)):
                            hits.append(s)
                    assert len(hits) == 1
                    sb = layout.boxes[hits[0]]
                    li = [g[d] - sb.origin[d] + sb.ng_lo[d] for d in range(3)]
                    a[kz, ky, kx] = arrays[hits[0]][li[2], li[1], li[0]]
        out.append(a)
    return out


@pytest.mark.parametrize("kind", ["local", "local_open", "hybrid", "independent"])
def test_exchange_matches_owner_search(O, kind):
    rng = np.random.default_rng(17)
    if kind == "local":
        lay = I.local_layout((12, 8, 8), (3, 2, 2), 2, 4)
    elif kind == "local_open":
        lay = I.local_layout((12, 8, 8), (3, 2, 2), 3, 4, periodic=(0, 1, 0))
    elif kind == "hybrid":
        lay = I.hybrid_layout((16, 6, 6), (2, 1, 1), 3, 4)
    else:
        lay = I.independent_layout(seed=3, nboxes=3, sizes=(8, 10, 12), ngs=(1, 2), min_interior=4)
    arrs = [rng.standard_normal(b.shape) for b in lay.boxes]
    got = O.exchange(lay, arrs)
    ref = _brute_exchange(lay, arrs)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


# ---------------------------------------------------------------------------
# Decompositions: local -> global as guards grow (Sec. 1.3)
# ---------------------------------------------------------------------------

def test_local_converges_to_global_with_guards(O):
    gsz, p, dt, steps = 32, 8, 0.9, 6
    f = I.laser_fields((gsz,) * 3, wavelength=8.0, waist=5.0, duration=4.0)
    glay = I.global_layout((gsz,) * 3, p)
    gref = O.push(glay, {k: I.scatter_global(v, glay) for k, v in f.items()}, {}, steps,
                  (1.0,) * 3, dt)
    errs = []
    for ng in (1, 2, 4, 8):
        lay = I.local_layout((gsz,) * 3, (2, 2, 2), ng, p)
        out = O.push(lay, {k: I.scatter_global(v, lay) for k, v in f.items()}, {}, steps,
                     (1.0,) * 3, dt)
        # compare interiors with the global solution
        ref = {k: I.scatter_global(gref[k][0], lay) for k in O.COMPS}
        errs.append(O.rel_l2_fields(lay, out, ref, O.COMPS))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 0.05 * errs[0]


def test_hybrid_single_group_equals_global(O):
    """A hybrid layout with one group on every axis is the global solver."""
    gsz = (16, 12, 10)
    f = I.laser_fields(gsz, wavelength=6.0, waist=3.0, duration=3.0)
    glay = I.global_layout(gsz, 8)
    hlay = I.hybrid_layout(gsz, (1, 1, 1), 4, 8)
    a = O.push(glay, {k: I.scatter_global(v, glay) for k, v in f.items()}, {}, 3, (1.0,) * 3, 0.8)
    b = O.push(hlay, {k: I.scatter_global(v, hlay) for k, v in f.items()}, {}, 3, (1.0,) * 3, 0.8)
    for k in O.COMPS:
        assert np.array_equal(a[k][0], b[k][0])


# ---------------------------------------------------------------------------
# Memory model (Sec. 2.2 eqs. (1)-(6), Sec. 2.3 eq. (7)): printed values
# ---------------------------------------------------------------------------

def _golden():
    rows = []
    with open(os.path.join(GOLDEN, "memory_model.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, d, nm, v = line.split()
                rows.append((name, int(d), int(nm), float(v)))
    return rows


def test_memory_model_printed_values(O):
    for name, d, nm, v in _golden():
        if name == "local_max":
            n, n_g = 4096.0, 16
            n_p = n / n_g                       # maximum processors: n/n_p = n_g
            assert abs(O.memory_local(n, n_p, n_g) / n ** 3 - v) < 1e-9
        elif name == "gain_limit":
            assert abs(O.memory_gain(d, 1e9) - v) < 1e-6
        elif name == "guard_gain":
            assert round(O.guard_gain(d, nm)) == v
            assert abs(O.guard_gain(d, nm) - 8 / 0.96) < 1e-12


def test_memory_gain_is_ratio_of_eqs_1_and_3(O):
    n, n_g = 1024.0, 8
    n_p = n / n_g
    for n_mpi in (1, 2, 4, 8, 32):
        ratio = O.memory_local(n, n_p, n_g) / O.memory_hybrid(n, n_p, n_g, n_mpi)
        assert abs(ratio - O.memory_gain(3, n_mpi)) < 1e-9 * ratio
        # eq. (4)
        assert abs(O.memory_hybrid(n, n_p, n_g, n_mpi) / n ** 3
                   - ((2 + n_mpi) / n_mpi) ** 3) < 1e-9
    assert abs(O.memory_gain(3, 1) - 1.0) < 1e-15


def test_workload_memory_ratio_local_vs_hybrid(O):
    """The one-GPU hybrid/local workloads: padded-cell ratio 18 = the d = 1
    gain at n_mpi = 4 (eq. (6)) times 3 x 3 for the two axes the group spans."""
    hyb = I.hybrid_layout((1024, 256, 256), (4, 1, 1), 64, 64)
    loc = I.local_layout((1024, 256, 256), (16, 4, 4), 64, 64)
    assert loc.cells / hyb.cells == 18.0
    assert abs(O.memory_gain(1, 4) * 9 - 18.0) < 1e-12


# ---------------------------------------------------------------------------
# Dual-grid coupling (Sec. 2.5.2): cell-by-cell owner search, round trip
# ---------------------------------------------------------------------------

def _brute_couple(src, arrays, dst):
    out = []
    for b in dst.boxes:
        a = np.zeros(b.shape)
        for kz in range(b.n[2]):
            for ky in range(b.n[1]):
                for kx in range(b.n[0]):
                    loc = (kx, ky, kz)
                    g = [b.origin[d] - b.ng_lo[d] + loc[d] for d in range(3)]
                    outside = False
                    for d in range(3):
                        if dst.periodic[d]:
                            g[d] %= dst.global_n[d]
                        elif not 0 <= g[d] < dst.global_n[d]:
                            outside = True
                    if outside:
                        continue
                    hits = [s for s, sb in enumerate(src.boxes)
                            if all(sb.origin[d] <= g[d] < sb.origin[d] + sb.interior[d] for d in range(3))]
                    assert len(hits) == 1
                    sb = src.boxes[hits[0]]
                    li = tuple(g[d] - sb.origin[d] + sb.ng_lo[d] for d in range(3))
                    a[kz, ky, kx] = arrays[hits[0]][li[2], li[1], li[0]]
        out.append(a)
    return out


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 0)])
def test_couple_matches_owner_search(O, periodic):
    rng = np.random.default_rng(19)
    g1 = I.local_layout((12, 8, 8), (3, 2, 2), 1, 4, periodic=periodic)      # particle grid, thin guards
    g2 = I.local_layout((12, 8, 8), (2, 1, 2), (2, 3, 2), 4, periodic=periodic)   # FFT grid, wide guards
    a1 = [rng.standard_normal(b.shape) for b in g1.boxes]
    got = O.couple(g1, a1, g2)
    for g, r in zip(got, _brute_couple(g1, a1, g2)):
        assert np.array_equal(g, r)
    a2 = [rng.standard_normal(b.shape) for b in g2.boxes]
    back = O.couple(g2, a2, g1)
    for g, r in zip(back, _brute_couple(g2, a2, g1)):
        assert np.array_equal(g, r)


def test_couple_round_trip_is_identity_on_consistent_fields(O):
    rng = np.random.default_rng(20)
    g1 = I.local_layout((16, 12, 8), (4, 3, 2), 1, 4)
    g2 = I.hybrid_layout((16, 12, 8), (2, 1, 1), 3, 4)
    a1 = O.exchange(g1, [rng.standard_normal(b.shape) for b in g1.boxes])
    a2 = O.couple(g1, a1, g2)
    assert all(np.array_equal(x, y) for x, y in zip(O.exchange(g2, a2), a2))   # G2 guards filled too
    for x, y in zip(O.couple(g2, a2, g1), a1):
        assert np.array_equal(x, y)


def test_couple_rejects_different_domains(O):
    with pytest.raises(ValueError):
        O.couple(I.local_layout((8, 8, 8), (2, 1, 1), 1, 4), [np.zeros((10, 10, 6))] * 2,
                 I.local_layout((8, 8, 12), (2, 1, 1), 1, 4))


# ---------------------------------------------------------------------------
# Nodal (collocated) variant: centred weights, symbol, conservation
# ---------------------------------------------------------------------------

def test_nodal_weights_low_orders_and_exactness(O):
    _same(O.nodal_weights(2), [Fraction(1)])
    _same(O.nodal_weights(4), [Fraction(4, 3), Fraction(-1, 3)])
    # the classical 4th-order centred coefficients 2/3 and -1/12 (beta_l / (2 l))
    b = O.nodal_weights(4)
    _same([b[0] / 2, b[1] / 4], [Fraction(2, 3), Fraction(-1, 12)])
    for p in (2, 4, 8, 16, 32):
        _exactness(O.nodal_weights(p), lambda l: l, p)
    assert O.nodal_weights(0) is None


def _centred_diff(f, axis, p, h):
    """Order-p centred difference on a periodic nodal grid, cell by cell, with
    weights from the exactness system sum_l beta_l l^(2j) = delta_j0 solved
    by exact elimination (independent of the oracle's Lagrange formula)."""
    q = p // 2
    A = [[Fraction(l ** (2 * j)) for l in range(1, q + 1)] + [Fraction(int(j == 0))] for j in range(q)]
    for c in range(q):                            # exact Gauss-Jordan over the rationals
        piv = next(r for r in range(c, q) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        for r in range(q):
            if r != c and A[r][c] != 0:
                fac = A[r][c] / A[c][c]
                A[r] = [a - fac * b for a, b in zip(A[r], A[c])]
    w = [float(A[r][q] / A[r][r]) for r in range(q)]   # beta_l
    out = np.zeros_like(f)
    for l, b in enumerate(w, start=1):
        out += b * (np.roll(f, -l, axis) - np.roll(f, l, axis)) / (2 * l * h)
    return out


@pytest.mark.parametrize("p", [2, 4, 8, 16])
def test_nodal_wavenumber_is_stencil_eigenvalue_and_order(O, p):
    n, h = 24, 0.7
    x = np.arange(n)
    for m in range(0, n // 2 + 1):
        k = 2 * np.pi * m / (n * h)
        f = np.exp(1j * k * x * h).reshape(1, 1, n)
        lam = (_centred_diff(f, 2, p, h) / f).ravel()
        assert np.allclose(lam, 1j * O.modified_wavenumber_nodal(k, h, p), atol=1e-11, rtol=0)
    e1 = abs(O.modified_wavenumber_nodal(0.2, 1.0, p) - 0.2)
    e2 = abs(O.modified_wavenumber_nodal(0.1, 1.0, p) - 0.1)
    if p <= 8:
        assert 2 ** (p + 1) * 0.8 < e1 / e2 < 2 ** (p + 1) * 1.2


def test_nodal_push_conserves_energy_and_div_b(O):
    rng = np.random.default_rng(31)
    n, p = 16, 8
    lay = I.global_layout((n, n, n), p)
    f = {k: [rng.standard_normal((n, n, n))] for k in O.COMPS}
    # a divergence-free B (curl of a random potential with the same centred stencil)
    A_ = [rng.standard_normal((n, n, n)) for _ in range(3)]
    dd = lambda a, ax: _centred_diff(a, ax, p, 1.0)
    f["Bx"] = [dd(A_[2], 1) - dd(A_[1], 0)]
    f["By"] = [dd(A_[0], 0) - dd(A_[2], 2)]
    f["Bz"] = [dd(A_[1], 2) - dd(A_[0], 1)]
    out = O.push(lay, f, {}, 5, (1.0,) * 3, 0.7, nodal=True)
    e0 = sum(float(np.sum(f[k][0] ** 2)) for k in O.COMPS)
    e1 = sum(float(np.sum(out[k][0] ** 2)) for k in O.COMPS)
    assert abs(e1 - e0) <= 1e-12 * e0
    divb = dd(out["Bx"][0], 2) + dd(out["By"][0], 1) + dd(out["Bz"][0], 0)
    assert np.abs(divb).max() <= 1e-11 * max(1.0, np.abs(out["Bx"][0]).max())


def test_nodal_plane_wave_dispersion(O):
    """A single transverse mode rotates with omega = c K_nodal per step."""
    n, p, dt, h = 16, 4, 0.6, 1.0
    lay = I.global_layout((n, n, n), p)
    m = 3
    k = 2 * np.pi * m / (n * h)
    x = np.arange(n) * h
    ey = np.cos(k * x)[None, None, :] * np.ones((n, n, 1))
    K = O.modified_wavenumber_nodal(k, h, p)
    bz = ey.copy()                                   # B = E / c for a +x wave with the nodal K
    f = {c: [np.zeros((n, n, n))] for c in O.COMPS}
    f["Ey"] = [ey]
    f["Bz"] = [bz]
    out = O.push(lay, f, {}, 1, (h,) * 3, dt, nodal=True)
    want = np.cos(k * x - K * dt)[None, None, :] * np.ones((n, n, 1))
    assert np.abs(out["Ey"][0] - want).max() <= 1e-12


def test_nodal_infinite_order_keeps_fields_real(O):
    """At p = infinity the collocated symbol is 0 at Nyquist; the push of a
    real field stays real (imaginary part of the inverse FFT at rounding)."""
    rng = np.random.default_rng(33)
    f = {k: rng.standard_normal((8, 10, 12)) for k in O.COMPS}
    K = O.modified_wavenumber_nodal(O.axis_wavenumbers(12, 1.0), 1.0, 0)
    assert K[6] == 0.0 and K[5] == O.axis_wavenumbers(12, 1.0)[5]
    _, imag = O.push_box(f, None, (1.0,) * 3, 0, 0.7, nodal=True, return_imag=True)
    assert imag <= 1e-13


# ---------------------------------------------------------------------------
# The two implementations against each other, and the FP32 rounding model
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["local_vacuum", "local_rho_inf", "hybrid_J", "independent_rho_nodal",
                                  "open_J_nodal"])
def test_cpp_and_numpy_oracles_agree(case):
    rng = np.random.default_rng(51)
    lay, form, nodal = {
        "local_vacuum": (I.local_layout((24, 16, 16), (2, 2, 1), 3, 8), "vacuum", False),
        "local_rho_inf": (I.local_layout((24, 16, 16), (2, 2, 1), 3, 0), "rho", False),
        "hybrid_J": (I.hybrid_layout((32, 12, 10), (2, 1, 1), 4, 4), "J", False),
        "independent_rho_nodal": (I.independent_layout(seed=3, nboxes=3, sizes=(8, 10, 12), ngs=(1, 2),
                                                       min_interior=4), "rho", True),
        "open_J_nodal": (I.local_layout((24, 16, 16), (2, 2, 1), 3, 8, periodic=(0, 1, 0)), "J", True),
    }[case]
    f = {k: psatd_oracle.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes])
         for k in psatd_oracle.COMPS}
    s = {k: psatd_oracle.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes])
         for k in ("Jx", "Jy", "Jz", "rho")}
    a = psatd_oracle.push(lay, f, s, 3, (1.0, 0.9, 1.1), 0.7, form=form, nodal=nodal)
    b = psatd_numpy.push(lay, f, s, 3, (1.0, 0.9, 1.1), 0.7, form=form, nodal=nodal)
    for k in a:
        for x, y in zip(a[k], b[k]):
            assert np.abs(x - y).max() <= 1e-13 * (1 + np.abs(y).max()), (case, k)


def test_fp32_rounding_model():
    """precision=32 runs the same steps in FP32: close to the FP64 push at the
    level of FP32 rounding, but not equal to it (it really rounds)."""
    rng = np.random.default_rng(52)
    lay = I.local_layout((32, 16, 16), (2, 1, 1), 4, 8)
    f = {k: psatd_oracle.exchange(lay, I.round_to([rng.standard_normal(b.shape) for b in lay.boxes], np.float32))
         for k in psatd_oracle.COMPS}
    a = psatd_oracle.push(lay, f, {}, 4, (1.0,) * 3, 0.9)
    b = psatd_oracle.push(lay, f, {}, 4, (1.0,) * 3, 0.9, precision=32)
    err = psatd_oracle.rel_l2_fields(lay, b, a, psatd_oracle.COMPS)
    assert 1e-8 < err < 2e-6, err
    for k in b:          # every value is an FP32 number
        for x in b[k]:
            assert np.array_equal(x, x.astype(np.float32).astype(np.float64))


# ---------------------------------------------------------------------------
# Absorbing layers (two-step split-field PML; the paper, end of Sec. 2.6,
# only names the method): the oracle's layers against closed forms
# ---------------------------------------------------------------------------

def _pulse_along_x(nx, ny, nz, x0=128.0, tau=10.0, lam=16.0):
    x = np.arange(nx)
    g = lambda xs: np.exp(-((xs - x0) / tau) ** 2) * np.cos(2 * np.pi / lam * (xs - x0))
    f = {k: np.zeros((nz, ny, nx)) for k in psatd_oracle.COMPS}
    f["Ey"][:] = g(x + 0.0)[None, None, :]          # E_y at (i, j + 1/2, k): x offset 0
    f["Bz"][:] = g(x + 0.5)[None, None, :]          # B_z at (i + 1/2, j + 1/2, k)
    return f


def test_pml_without_conductivity_is_the_plain_push():
    rng = np.random.default_rng(61)
    lay = I.local_layout((32, 16, 16), (2, 1, 1), 4, 8)
    f = {k: psatd_oracle.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes])
         for k in psatd_oracle.COMPS}
    a = psatd_oracle.push(lay, f, {}, 3, (1.0,) * 3, 0.7)
    b = psatd_oracle.push(lay, f, {}, 3, (1.0,) * 3, 0.7,
                          pml=dict(width=(6, 4, 0), sigma_max=(0.0, 0.0, 0.0), order=2))
    for k in psatd_oracle.COMPS:
        for x, y in zip(a[k], b[k]):
            assert np.abs(x - y).max() <= 1e-13 * (1 + np.abs(y).max())


@pytest.mark.parametrize("smax,order,p", [(0.1875, 2, 0), (0.09375, 2, 16), (0.25, 3, 0)])
def test_pml_normal_incidence_transmission_and_reflection(smax, order, p):
    """A pulse along +x in a periodic 256-cell box with layers of w = 32 cells
    on both x faces: after one lap (it crosses both layers) its amplitude is
    exp(-int s dx / c) = exp(-2 s_max w / (c (m + 1))), the attenuation of a
    continuous matched layer at normal incidence; a continuous PML reflects
    nothing, so the field left behind the pulse once it is inside the layer
    stays at the discretisation level; the energy never grows."""
    nx, w, dt = 256, 32, 0.5
    lay = I.global_layout((nx, 4, 4), p)
    f0 = _pulse_along_x(nx, 4, 4)
    cur = {k: [v] for k, v in f0.items()}
    pml = dict(width=(w, 0, 0), sigma_max=(smax, 0.0, 0.0), order=order)
    e_prev = sum(float(np.sum(v ** 2)) for v in f0.values())
    refl = None
    for s in range(int(256 / dt)):
        cur = psatd_oracle.push(lay, cur, {}, 1, (1.0,) * 3, dt, pml=pml)
        e = sum(float(np.sum(cur[k][0] ** 2)) for k in psatd_oracle.COMPS)
        assert e <= e_prev * (1 + 1e-12)
        e_prev = e
        if (s + 1) * dt == 112:          # pulse centre at x = 240, inside the high-x layer
            ey = cur["Ey"][0][0, 0]
            refl = float(np.sqrt(np.sum(ey[40:200] ** 2) / np.sum(f0["Ey"][0, 0] ** 2)))
    amp = float(np.abs(cur["Ey"][0][0, 0]).max())
    ana = math.exp(-2 * smax * w / (order + 1))
    assert abs(amp / ana - 1) < 0.01, (amp, ana)
    assert refl < 1e-5, refl


def test_pml_split_parts_sum_to_the_fields():
    """A wave along x has d/dy = d/dz = 0: started with the whole of B_z in
    its x part (B_zx = B_z) and E_y in its x part (E_yz = 0), the y part of
    B_z and the z part of E_y must stay exactly 0 in and outside the layers,
    i.e. the stored parts keep summing to the components."""
    nx = 64
    lay = I.global_layout((nx, 8, 8), 8)
    f0 = _pulse_along_x(nx, 8, 8, x0=40.0, tau=4.0, lam=8.0)
    cur = {k: [v] for k, v in f0.items()}
    cur["Bzx"] = [f0["Bz"].copy()]
    pml = dict(width=(8, 0, 0), sigma_max=(0.5, 0.0, 0.0), order=2)
    for _ in range(40):
        cur = psatd_oracle.push(lay, cur, {}, 1, (1.0,) * 3, 0.5, pml=pml)
    scale = np.abs(f0["Bz"]).max()
    assert np.abs(cur["Bz"][0] - cur["Bzx"][0]).max() < 1e-12 * scale
    assert np.abs(cur["Eyz"][0]).max() < 1e-12 * scale
