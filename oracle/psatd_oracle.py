"""FP64 reference implementation ("oracle") of the PSATD Maxwell push:
Python interface to liboracle.so, built from oracle/psatd_oracle.cpp (plain
C++, its own mixed-radix FFT, OpenMP over FFT lines and modes).

TEST INFRASTRUCTURE.  Only the test-suite, the smoke check of the package
entry point and the CPU-baseline leg of the benchmark import this module.  The
product path (the CUDA library and its Python binding) never imports it, and
this module imports nothing from the product package.

The method (paper Sec. 1.1 for PSATD, Sec. 1.3 and Fig. 1 for the local
decomposition, Sec. 2.1 for the hybrid one), the readings of what the paper
leaves unsaid (update equations, stencil, Yee positions, Fourier convention)
and the FFT are stated in psatd_oracle.cpp.  This module only moves arrays
in and out; the helpers that are not arithmetic of the method (error
metrics, interior slices) and the paper's memory model (Sec. 2.2 eqs. (1)-(6),
Sec. 2.3 eq. (7)) are plain Python.

Array conventions: a box's array has shape (n_z, n_y, n_x) (x fastest in
memory); a field is a dict component -> list of per-box arrays.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "psatd_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

# Yee offsets (cells) of every component: E and J on edges, B on faces,
# rho on nodes (the order of the C++ table).
YEE = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Bx": (0.0, 0.5, 0.5), "By": (0.5, 0.0, 0.5), "Bz": (0.5, 0.5, 0.0),
    "Jx": (0.5, 0.0, 0.0), "Jy": (0.0, 0.5, 0.0), "Jz": (0.0, 0.0, 0.5),
    "rho": (0.0, 0.0, 0.0),
}
COMPS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
_FORMS = {"vacuum": 0, "J": 1, "rho": 2}
_KINDS = {"global": 0, "local": 1, "hybrid": 2, "independent": 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (g++ -O2 -fopenmp)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, SRC]
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)          # no OpenMP runtime: one thread
    os.replace(tmp, LIB)
    return LIB


class _Box(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("ng_lo", ctypes.c_int32 * 3), ("ng_hi", ctypes.c_int32 * 3),
                ("origin", ctypes.c_int64 * 3), ("p", ctypes.c_int32)]


class _Pml(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32 * 3), ("sigma_max", ctypes.c_double * 3), ("order", ctypes.c_int32)]


# the stored split part of every component in the PML (the other part is the
# component minus it): E_x along y, E_y along z, E_z along x, same for B
SPLIT = ("Exy", "Eyz", "Ezx", "Bxy", "Byz", "Bzx")


class _Layout(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("global_n", ctypes.c_int32 * 3), ("periodic", ctypes.c_int32 * 3),
                ("nbox", ctypes.c_int32), ("boxes", ctypes.POINTER(_Box))]


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        lib.oracle_threads.restype = I32
        lib.oracle_fft3.argtypes = [I32, I32, I32, I32, I32, P]
        lib.oracle_weights.argtypes = [I32, I32, P]
        lib.oracle_modified_wavenumber.argtypes = [I64, P, D, I32, I32, P]
        lib.oracle_coefficients.argtypes = [I64, P, D, D, P, P, P, P]
        lib.oracle_update_modes.argtypes = [I64, PP, PP, PP, P, PP, D, D, D, I32]
        lib.oracle_exchange.argtypes = [ctypes.POINTER(_Layout), P]
        lib.oracle_couple.argtypes = [ctypes.POINTER(_Layout), P, ctypes.POINTER(_Layout), P]
        lib.oracle_push.argtypes = [ctypes.POINTER(_Layout), PP, PP, P, I32, P, D, D, D, I32, I32, I32, P,
                                    ctypes.POINTER(_Pml), PP]
        for f in ("oracle_fft3", "oracle_weights", "oracle_modified_wavenumber", "oracle_coefficients",
                  "oracle_update_modes", "oracle_exchange", "oracle_couple", "oracle_push"):
            getattr(lib, f).restype = I32
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else every core)."""
    return int(_L().oracle_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle: {what} failed (code {rc})")


# ----------------------------------------------------------------------------
# FFT
# ----------------------------------------------------------------------------

def fft3(a):
    """Unnormalised forward 3D DFT of an (n_z, n_y, n_x) array."""
    x = np.array(a, dtype=np.complex128, order="C", copy=True)
    nz, ny, nx = x.shape
    _check(_L().oracle_fft3(nx, ny, nz, -1, 64, _ptr(x)), "fft3")
    return x


def ifft3(a):
    """Inverse 3D DFT with the 1/N factor."""
    x = np.array(a, dtype=np.complex128, order="C", copy=True)
    nz, ny, nx = x.shape
    _check(_L().oracle_fft3(nx, ny, nz, 1, 64, _ptr(x)), "ifft3")
    return x / x.size


def fft3_f32(a):
    """The same forward transform in FP32 arithmetic (the rounding model)."""
    x = np.array(a, dtype=np.complex64, order="C", copy=True)
    nz, ny, nx = x.shape
    _check(_L().oracle_fft3(nx, ny, nz, -1, 32, _ptr(x)), "fft3")
    return x


# ----------------------------------------------------------------------------
# Stencil, wavenumbers, coefficients, per-mode update
# ----------------------------------------------------------------------------

def _weights(p, nodal):
    if p == 0:
        return None
    if p < 2 or p % 2:
        raise ValueError("order p must be even and >= 2, or 0 for infinite")
    out = np.zeros(p // 2)
    _check(_L().oracle_weights(p, int(nodal), _ptr(out)), "weights")
    return [float(v) for v in out]


def stencil_weights(p: int):
    """alpha_l, l = 1..p/2, of the order-p staggered difference (floats);
    None for infinite order (p = 0)."""
    return _weights(p, False)


def nodal_weights(p: int):
    """beta_l, l = 1..p/2, of the order-p centred nodal difference."""
    return _weights(p, True)


def _mw(k, h, p, nodal):
    k = np.asarray(k, dtype=np.float64)
    flat = np.ascontiguousarray(k.ravel())
    out = np.zeros_like(flat)
    _check(_L().oracle_modified_wavenumber(flat.size, _ptr(flat), float(h), int(p), int(nodal), _ptr(out)),
           "modified_wavenumber")
    out = out.reshape(k.shape)
    return float(out) if out.ndim == 0 else out


def modified_wavenumber(k, h: float, p: int):
    """Fourier symbol K(k) of the order-p staggered difference."""
    return _mw(k, h, p, False)


def modified_wavenumber_nodal(k, h: float, p: int):
    """Fourier symbol K(k) of the order-p centred nodal difference (K = 0 at
    the Nyquist wavenumber for infinite order)."""
    return _mw(k, h, p, True)


def axis_wavenumbers(n: int, h: float):
    """True wavenumber of every index of an n-point periodic axis."""
    m = np.arange(n)
    mt = np.where(m <= n // 2, m, m - n)
    return 2.0 * np.pi * mt / (n * h)


def coefficients(K2, c: float, dt: float):
    """C, Sw, X1, X3 as functions of K^2."""
    K2 = np.ascontiguousarray(np.asarray(K2, dtype=np.float64).ravel())
    outs = [np.zeros_like(K2) for _ in range(4)]
    _check(_L().oracle_coefficients(K2.size, _ptr(K2), float(c), float(dt), *[_ptr(o) for o in outs]),
           "coefficients")
    return tuple(outs)


def _pp(arrs):
    return (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])


def update_modes(E, B, J, R, K, dt, c=1.0, eps0=1.0, form="vacuum"):
    """Advance centred spectra by one step (3-tuples of complex arrays E, B,
    J or None, R or None; K a 3-tuple of real arrays).  Returns (E', B', R')."""
    shape = np.broadcast(*E, *B, *K).shape
    cv = lambda a: np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.complex128).ravel().copy()
    rv = lambda a: np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.float64).ravel().copy()
    e = [cv(x) for x in E]
    b = [cv(x) for x in B]
    j = [cv(x) for x in J] if J is not None and form != "vacuum" else None
    r = cv(R) if form == "rho" else None
    k = [rv(x) for x in K]
    n = e[0].size
    _check(_L().oracle_update_modes(n, _pp(e), _pp(b), _pp(j) if j else None, _ptr(r) if r is not None else None,
                                    _pp(k), float(dt), float(c), float(eps0), _FORMS[form]), "update_modes")
    En = tuple(x.reshape(shape) for x in e)
    Bn = tuple(x.reshape(shape) for x in b)
    return En, Bn, (r.reshape(shape) if r is not None else None)


# ----------------------------------------------------------------------------
# Layouts, push, exchange, coupling
# ----------------------------------------------------------------------------

def _layout(layout):
    nb = len(layout.boxes)
    arr = (_Box * nb)()
    for i, b in enumerate(layout.boxes):
        arr[i].n[:] = list(b.n)
        arr[i].ng_lo[:] = list(b.ng_lo)
        arr[i].ng_hi[:] = list(b.ng_hi)
        arr[i].origin[:] = list(b.origin)
        arr[i].p = int(b.p)
    L = _Layout()
    L.kind = _KINDS[layout.kind]
    L.global_n[:] = [int(v) for v in layout.global_n]
    L.periodic[:] = [int(v) for v in layout.periodic]
    L.nbox = nb
    L.boxes = ctypes.cast(arr, ctypes.POINTER(_Box))
    L._keep = arr
    return L


def _pack(layout, arrays):
    return np.concatenate([np.ascontiguousarray(a, dtype=np.float64).ravel() for a in arrays]) \
        if arrays else np.zeros(0)


def _unpack(layout, flat):
    out, off = [], 0
    for b in layout.boxes:
        n = b.n[0] * b.n[1] * b.n[2]
        out.append(flat[off:off + n].reshape(b.n[2], b.n[1], b.n[0]).copy())
        off += n
    return out


def exchange(layout, arrays):
    """New per-box arrays whose guards hold the owning interior values."""
    L = _layout(layout)
    flat = _pack(layout, arrays)
    _check(_L().oracle_exchange(ctypes.byref(L), _ptr(flat)), "exchange (interiors must tile the domain)")
    return _unpack(layout, flat)


def couple(src_layout, src_arrays, dst_layout):
    """Dual-grid coupling (paper Sec. 2.5.2): every destination cell takes the
    source interior cell with the same global index."""
    S, Dl = _layout(src_layout), _layout(dst_layout)
    flat = _pack(src_layout, src_arrays)
    n = sum(b.n[0] * b.n[1] * b.n[2] for b in dst_layout.boxes)
    out = np.zeros(n)
    rc = _L().oracle_couple(ctypes.byref(S), _ptr(flat), ctypes.byref(Dl), _ptr(out))
    if rc == 3:
        raise ValueError("layouts of different domains")
    _check(rc, "couple")
    return _unpack(dst_layout, out)


def push(layout, fields, src, nsteps, h, dt, c=1.0, eps0=1.0, form="vacuum", boxes=None, nodal=False,
         precision=64, return_imag=False, pml=None):
    """Advance ``fields`` (dict comp -> list of per-box arrays) by ``nsteps``
    steps: every step advances each box, then exchanges guards.  With form
    'rho', ``src['rho']`` is advanced too and returned in the output dict.
    ``boxes`` restricts the advance to a subset (no exchange then).
    precision 32 runs the FP32 rounding model instead of the oracle.

    pml: absorbing layers, dict(width=(wx, wy, wz), sigma_max=(sx, sy, sz),
    order=m); the stored split parts are read from ``fields[SPLIT[i]]`` when
    present (else zero) and returned in the output dict (vacuum form)."""
    L = _layout(layout)
    f = [_pack(layout, fields[k]) for k in COMPS]
    s = None
    if form in ("J", "rho"):
        s = [_pack(layout, src[k]) for k in ("Jx", "Jy", "Jz")]
        s.append(_pack(layout, src["rho"]) if form == "rho" else np.zeros(1))
    mask = None
    if boxes is not None:
        mask = np.zeros(len(layout.boxes), np.uint8)
        mask[list(boxes)] = 1
    imag = np.zeros(1)
    hh = np.asarray(h, dtype=np.float64)
    pm, sp = None, None
    if pml is not None:
        pm = _Pml()
        pm.width[:] = [int(v) for v in pml["width"]]
        pm.sigma_max[:] = [float(v) for v in pml["sigma_max"]]
        pm.order = int(pml["order"])
        sp = [_pack(layout, fields[k]) if k in fields else np.zeros(f[0].size) for k in SPLIT]
    rc = _L().oracle_push(ctypes.byref(L), _pp(f), _pp(s) if s else None,
                          _ptr(mask) if mask is not None else None, int(nsteps), _ptr(hh), float(dt), float(c),
                          float(eps0), _FORMS[form], int(nodal), int(precision), _ptr(imag),
                          ctypes.byref(pm) if pm is not None else None, _pp(sp) if sp else None)
    _check(rc, "push")
    out = {k: _unpack(layout, a) for k, a in zip(COMPS, f)}
    if sp:
        out.update({k: _unpack(layout, a) for k, a in zip(SPLIT, sp)})
    if form == "rho":
        out["rho"] = _unpack(layout, s[3])
    if return_imag:
        return out, float(imag[0])
    return out


class _OneBox:
    def __init__(self, shape, p):
        self.n = (shape[2], shape[1], shape[0])
        self.ng_lo = self.ng_hi = (0, 0, 0)
        self.origin = (0, 0, 0)
        self.p = p


class _OneLayout:
    def __init__(self, shape, p):
        self.kind = "independent"
        self.global_n = (0, 0, 0)
        self.periodic = (1, 1, 1)
        self.boxes = [_OneBox(shape, p)]


def push_box(f, src, h, p, dt, c=1.0, eps0=1.0, form="vacuum", return_imag=False, nodal=False, precision=64):
    """One PSATD step of one periodic box.  f: dict Ex..Bz -> (nz, ny, nx)
    arrays; src: dict Jx, Jy, Jz[, rho] or None.  Returns a new dict (with
    'rho' in the rho form), and the largest imaginary part of the inverse
    transforms when return_imag."""
    lay = _OneLayout(f["Ex"].shape, p)
    fl = {k: [f[k]] for k in COMPS}
    sl = {k: [v] for k, v in src.items()} if src else {}
    out, imag = push(lay, fl, sl, 1, h, dt, c, eps0, form, nodal=nodal, precision=precision, return_imag=True)
    out = {k: v[0] for k, v in out.items()}
    return (out, imag) if return_imag else out


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

def _interior_slices(box):
    return tuple(slice(box.ng_lo[d], box.n[d] - box.ng_hi[d]) for d in (2, 1, 0))


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
