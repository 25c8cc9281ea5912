"""Seeded synthetic inputs for the PSATD push: box layouts and initial fields.

This module produces *inputs only*.  It holds none of the solver's arithmetic
(no k-space update, no modified wavenumbers, no guard exchange of solver
state); it is the one module that both the FP64 oracle tests and the GPU path
consume, so that both sides see bit-identical inputs.

Layouts (the sub-domain / group geometry of the paper's Fig. 1):

* ``global``      one periodic box covering the whole domain (Sec. 1.2).
* ``local``       Cartesian sub-domains, each padded with ``ng`` guard cells on
                  every face (Fig. 1a, Sec. 1.3).
* ``hybrid``      groups of sub-domains; guards only on group faces that are
                  not periodic inside the group FFT (Fig. 1b, Sec. 2.1).
* ``independent`` boxes that are their own periodic domain; guards wrap onto
                  the box's own interior (uneven batch workload).

Arrays are numpy ``float64`` with shape ``(nz, ny, nx)`` (x fastest), one
array per field component and per box.

Field samples follow the Yee layout: E_x at (i+1/2, j, k), E_y at
(i, j+1/2, k), E_z at (i, j, k+1/2), B_x at (i, j+1/2, k+1/2), B_y at
(i+1/2, j, k+1/2), B_z at (i+1/2, j+1/2, k); J like E; rho at (i, j, k).

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64), which
is bit-reproducible across x86_64 and aarch64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
SOURCES = ("Jx", "Jy", "Jz", "rho")

# Sampling positions (in cells) used to evaluate analytic initial data.
_SAMPLE_AT = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Bx": (0.0, 0.5, 0.5), "By": (0.5, 0.0, 0.5), "Bz": (0.5, 0.5, 0.0),
    "Jx": (0.5, 0.0, 0.0), "Jy": (0.0, 0.5, 0.0), "Jz": (0.0, 0.0, 0.5),
    "rho": (0.0, 0.0, 0.0),
}


@dataclasses.dataclass(frozen=True)
class Box:
    """One FFT box: ``n`` cells per axis including guards (x, y, z order)."""
    n: Tuple[int, int, int]
    ng_lo: Tuple[int, int, int]
    ng_hi: Tuple[int, int, int]
    origin: Tuple[int, int, int]   # global index of the first interior cell
    p: int                         # stencil order (even >= 2) or 0 = infinite

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def interior(self):
        return tuple(self.n[d] - self.ng_lo[d] - self.ng_hi[d] for d in range(3))

    @property
    def cells(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def interior_cells(self):
        i = self.interior
        return i[0] * i[1] * i[2]


@dataclasses.dataclass
class Layout:
    kind: str                       # global | local | hybrid | independent
    global_n: Tuple[int, int, int]
    periodic: Tuple[int, int, int]
    boxes: List[Box]

    @property
    def cells(self):
        return sum(b.cells for b in self.boxes)

    @property
    def interior_cells(self):
        return sum(b.interior_cells for b in self.boxes)

    @property
    def guard_cells(self):
        return self.cells - self.interior_cells


def global_layout(n: Sequence[int], p: int, periodic=(1, 1, 1)) -> Layout:
    n = tuple(int(v) for v in n)
    return Layout("global", n, tuple(periodic),
                  [Box(n, (0, 0, 0), (0, 0, 0), (0, 0, 0), int(p))])


def local_layout(global_n, nsub, ng, p, periodic=(1, 1, 1)) -> Layout:
    """Cartesian split into nsub[d] sub-domains per axis, ng guards per face.
    Boxes are enumerated x fastest."""
    global_n = tuple(int(v) for v in global_n)
    nsub = tuple(int(v) for v in nsub)
    ng = tuple([int(ng)] * 3) if np.isscalar(ng) else tuple(int(v) for v in ng)
    inner = []
    for d in range(3):
        if global_n[d] % nsub[d]:
            raise ValueError("global size not divisible by sub-domain count")
        inner.append(global_n[d] // nsub[d])
    boxes = []
    for k in range(nsub[2]):
        for j in range(nsub[1]):
            for i in range(nsub[0]):
                idx = (i, j, k)
                n = tuple(inner[d] + 2 * ng[d] for d in range(3))
                org = tuple(idx[d] * inner[d] for d in range(3))
                boxes.append(Box(n, ng, ng, org, int(p)))
    return Layout("local", global_n, tuple(periodic), boxes)


def hybrid_layout(global_n, ngroups, ng, p, periodic=(1, 1, 1)) -> Layout:
    """Groups of sub-domains (Fig. 1b): ngroups[d] groups per axis.  An axis
    with a single group is periodic inside the group FFT and carries no
    guards; every split axis gets ng guards per face."""
    global_n = tuple(int(v) for v in global_n)
    ngroups = tuple(int(v) for v in ngroups)
    g = tuple(int(ng) if ngroups[d] > 1 or not periodic[d] else 0 for d in range(3))
    inner = [global_n[d] // ngroups[d] for d in range(3)]
    boxes = []
    for k in range(ngroups[2]):
        for j in range(ngroups[1]):
            for i in range(ngroups[0]):
                idx = (i, j, k)
                n = tuple(inner[d] + 2 * g[d] for d in range(3))
                org = tuple(idx[d] * inner[d] for d in range(3))
                boxes.append(Box(n, g, g, org, int(p)))
    return Layout("hybrid", global_n, tuple(periodic), boxes)


def independent_layout(seed=5, nboxes=300, sizes=(48, 60, 80, 96, 120),
                       ngs=(8, 24, 40), orders=(8, 16, 32, 0),
                       min_interior=16) -> Layout:
    """Uneven batch of self-periodic boxes.  Each axis size is drawn from
    ``sizes``; one guard width per box is drawn among the values of ``ngs``
    that leave at least ``min_interior`` interior cells on every axis; the
    stencil order is drawn from ``orders`` (0 = infinite)."""
    rng = np.random.default_rng(seed)
    boxes = []
    for _ in range(nboxes):
        n = tuple(int(v) for v in rng.choice(sizes, size=3))
        ok = [g for g in ngs if min(n) - 2 * g >= min_interior]
        ng = int(rng.choice(ok))
        p = int(rng.choice(orders))
        boxes.append(Box(n, (ng,) * 3, (ng,) * 3, (0, 0, 0), p))
    return Layout("independent", (0, 0, 0), (1, 1, 1), boxes)


# ----------------------------------------------------------------------------
# Scattering global data into padded boxes (plain periodic indexing)
# ----------------------------------------------------------------------------

def _box_index(box: Box, layout: Layout, d: int):
    """Global source index for every local cell of ``box`` along axis d, or -1
    where the cell lies outside a non-periodic domain."""
    if layout.kind == "independent":
        m = box.interior[d]
        return (np.arange(box.n[d]) - box.ng_lo[d]) % m
    N = layout.global_n[d]
    g = box.origin[d] - box.ng_lo[d] + np.arange(box.n[d])
    if layout.periodic[d]:
        return g % N
    return np.where((g >= 0) & (g < N), g, -1)


def scatter_global(arr: np.ndarray, layout: Layout) -> List[np.ndarray]:
    """Sample a global (nz, ny, nx) array at every padded cell of every box."""
    out = []
    for b in layout.boxes:
        ix, iy, iz = (_box_index(b, layout, d) for d in range(3))
        pad = np.concatenate([arr, np.zeros_like(arr[:1])], axis=0)
        pad = np.concatenate([pad, np.zeros_like(pad[:, :1])], axis=1)
        pad = np.concatenate([pad, np.zeros_like(pad[:, :, :1])], axis=2)
        # index -1 addresses the appended zero plane
        out.append(np.ascontiguousarray(pad[np.ix_(iz, iy, ix)]))
    return out


def scatter_self(interiors: List[np.ndarray], layout: Layout) -> List[np.ndarray]:
    """Independent boxes: wrap each box's own interior into its guards."""
    out = []
    for b, a in zip(layout.boxes, interiors):
        ix, iy, iz = (_box_index(b, layout, d) for d in range(3))
        out.append(np.ascontiguousarray(a[np.ix_(iz, iy, ix)]))
    return out


def zeros(layout: Layout) -> List[np.ndarray]:
    return [np.zeros(b.shape) for b in layout.boxes]


# ----------------------------------------------------------------------------
# Initial data
# ----------------------------------------------------------------------------

def _coords(n, comp, h=(1.0, 1.0, 1.0), shift=(0, 0, 0)):
    s = _SAMPLE_AT[comp]
    x = (np.arange(n[0]) + shift[0] + s[0]) * h[0]
    y = (np.arange(n[1]) + shift[1] + s[1]) * h[1]
    z = (np.arange(n[2]) + shift[2] + s[2]) * h[2]
    return np.meshgrid(z, y, x, indexing="ij")   # (Z, Y, X)


def plane_wave_set(seed=1, nwaves=8, mmax=6):
    """``nwaves`` transverse plane waves: integer wave-vector m in
    [-mmax, mmax]^3 \\ {0}, polarisation a seeded unit vector orthogonal to m,
    amplitude ~ N(0, 1), zero phase."""
    rng = np.random.default_rng(seed)
    waves = []
    while len(waves) < nwaves:
        m = rng.integers(-mmax, mmax + 1, size=3)
        if not m.any():
            continue
        v = rng.standard_normal(3)
        u = m / np.linalg.norm(m)
        e = v - np.dot(v, u) * u
        e /= np.linalg.norm(e)
        a = rng.standard_normal()
        waves.append((m.astype(np.int64), e, float(a)))
    return waves


def plane_wave_fields(waves, n, h=(1.0, 1.0, 1.0), c=1.0, t=0.0):
    """E = sum A e cos(k.x - c|k| t), B = (k_hat x E)/c on a periodic grid of
    n cells (k = 2 pi m / L), each component sampled at its Yee position."""
    L = [n[d] * h[d] for d in range(3)]
    out = {}
    for comp in COMPONENTS:
        Z, Y, X = _coords(n, comp, h)
        f = np.zeros((n[2], n[1], n[0]))
        for m, e, a in waves:
            k = np.array([2 * np.pi * m[d] / L[d] for d in range(3)])
            kn = np.linalg.norm(k)
            phase = k[0] * X + k[1] * Y + k[2] * Z - c * kn * t
            if comp[0] == "E":
                amp = a * e["xyz".index(comp[1])]
            else:
                b = np.cross(k / kn, e) * a / c
                amp = b["xyz".index(comp[1])]
            f += amp * np.cos(phase)
        out[comp] = f
    return out


def laser_fields(global_n, h=(1.0, 1.0, 1.0), c=1.0, wavelength=16.0,
                 waist=32.0, duration=20.0):
    """Gaussian laser pulse travelling along +x, centred in the domain:
    E_y = exp(-r^2/w0^2) exp(-(x-x0)^2/tau^2) cos(k0 (x-x0)), B_z = E_y / c,
    lengths in cells (1/e field half-widths)."""
    n = global_n
    x0, y0, z0 = (n[0] * h[0] / 2, n[1] * h[1] / 2, n[2] * h[2] / 2)
    k0 = 2 * np.pi / (wavelength * h[0])
    w0, tau = waist * h[1], duration * h[0]
    out = {c_: np.zeros((n[2], n[1], n[0])) for c_ in COMPONENTS}
    for comp in ("Ey", "Bz"):
        s = _SAMPLE_AT[comp]
        x = (np.arange(n[0]) + s[0]) * h[0] - x0
        y = (np.arange(n[1]) + s[1]) * h[1] - y0
        z = (np.arange(n[2]) + s[2]) * h[2] - z0
        fx = np.exp(-x ** 2 / tau ** 2) * np.cos(k0 * x)
        fy = np.exp(-y ** 2 / w0 ** 2)
        fz = np.exp(-z ** 2 / w0 ** 2)
        f = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
        out[comp] = f if comp == "Ey" else f / c
    return out


def laser_box_factors(layout: Layout, h=(1.0, 1.0, 1.0), c=1.0, wavelength=16.0,
                      waist=32.0, duration=20.0):
    """The laser of ``laser_fields`` is separable: per box and component return
    the 1D factors (fz, fy, fx) and the divisor d such that
    (fz[:,None,None] * fy[None,:,None] * fx[None,None,:]) / d equals
    ``scatter_global(laser_fields(...), layout)`` for that box, bit for bit.
    Components other than E_y and B_z are zero (returned as None)."""
    n = layout.global_n
    x0, y0, z0 = (n[0] * h[0] / 2, n[1] * h[1] / 2, n[2] * h[2] / 2)
    k0 = 2 * np.pi / (wavelength * h[0])
    w0, tau = waist * h[1], duration * h[0]
    out = {c_: None for c_ in COMPONENTS}
    for comp in ("Ey", "Bz"):
        s = _SAMPLE_AT[comp]
        x = (np.arange(n[0]) + s[0]) * h[0] - x0
        y = (np.arange(n[1]) + s[1]) * h[1] - y0
        z = (np.arange(n[2]) + s[2]) * h[2] - z0
        g = [np.append(np.exp(-x ** 2 / tau ** 2) * np.cos(k0 * x), 0.0),
             np.append(np.exp(-y ** 2 / w0 ** 2), 0.0),
             np.append(np.exp(-z ** 2 / w0 ** 2), 0.0)]
        per = []
        for b in layout.boxes:
            idx = [_box_index(b, layout, d) for d in range(3)]   # -1 -> appended 0
            per.append((g[2][idx[2]], g[1][idx[1]], g[0][idx[0]], 1.0 if comp == "Ey" else c))
        out[comp] = per
    return out


def _true_k2(n, h):
    ks = [2 * np.pi * np.fft.fftfreq(n[d], d=h[d]) for d in range(3)]
    KZ, KY, KX = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
    return KX ** 2 + KY ** 2 + KZ ** 2


def gaussian_filtered_current(n, h=(1.0, 1.0, 1.0), seed=2, sigma_frac=0.25):
    """J ~ N(0,1) per component and cell, multiplied in k-space by
    exp(-|k|^2 / (2 sigma^2)), sigma = sigma_frac * pi / h (true |k|)."""
    rng = np.random.default_rng(seed)
    sigma = sigma_frac * np.pi / min(h)
    g = np.exp(-_true_k2(n, h) / (2 * sigma ** 2))
    out = {}
    for comp in ("Jx", "Jy", "Jz"):
        r = rng.standard_normal((n[2], n[1], n[0]))
        out[comp] = np.fft.ifftn(np.fft.fftn(r) * g).real
    return out


def band_limited_current(n, rng, h=(1.0, 1.0, 1.0), kcut_frac=0.5):
    """J ~ N(0,1) per component and cell, keeping only |k| < kcut_frac*pi/h."""
    kc = kcut_frac * np.pi / min(h)
    mask = _true_k2(n, h) < kc ** 2
    out = {}
    for comp in ("Jx", "Jy", "Jz"):
        r = rng.standard_normal((n[2], n[1], n[0]))
        out[comp] = np.fft.ifftn(np.fft.fftn(r) * mask).real
    return out


def round_to(arrs, dtype):
    """Round every array to ``dtype`` and back to float64 (the FP32 runs are
    compared with an oracle fed the same rounded inputs)."""
    if isinstance(arrs, dict):
        return {k: round_to(v, dtype) for k, v in arrs.items()}
    if isinstance(arrs, list):
        return [round_to(a, dtype) for a in arrs]
    return np.asarray(arrs).astype(dtype).astype(np.float64)


# ----------------------------------------------------------------------------
# The five benchmark workloads (sizes from the paper's scaling discussion,
# Sec. 2.2-2.4, made concrete for one GPU)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    layout: Layout
    h: Tuple[float, float, float]
    dt: float
    c: float
    eps0: float
    steps: int
    sources: str          # 'vacuum' | 'rho'
    fields: Dict[str, List[np.ndarray]]
    src: Dict[str, List[np.ndarray]]


def make_workload(name: str, scale: int = 1, steps: int | None = None) -> Workload:
    """Build one of the five synthetic workloads.

    ``scale`` > 1 shrinks the spatial sizes (test-sized variant with the same
    structure): grid sizes and guard widths are divided by ``scale``.
    """
    h = (1.0, 1.0, 1.0)
    if name == "plane_waves_32":
        n = 32 // scale if scale > 1 else 32
        lay = global_layout((n, n, n), 0)
        waves = plane_wave_set(seed=1, mmax=min(6, n // 2 - 2))
        f = plane_wave_fields(waves, (n, n, n), h, 1.0, 0.0)
        fields = {k: scatter_global(v, lay) for k, v in f.items()}
        return Workload(name, lay, h, 0.5, 1.0, 1.0, steps or 64, "vacuum", fields, {})
    if name == "sources_128":
        n = 128 // scale
        lay = global_layout((n, n, n), 16)
        j = gaussian_filtered_current((n, n, n), h, seed=2)
        fields = {k: zeros(lay) for k in COMPONENTS}
        src = {k: scatter_global(v, lay) for k, v in j.items()}
        src["rho"] = zeros(lay)
        return Workload(name, lay, h, 0.9, 1.0, 1.0, steps or 200, "rho", fields, src)
    if name == "local_512":
        g = 512 // scale
        ng = max(16 // scale, 2)
        lay = local_layout((g, g, g), (8, 8, 8), ng, 32 // scale if scale > 1 else 32)
        f = laser_fields((g, g, g), h, 1.0, wavelength=16.0 / scale,
                         waist=32.0 / scale, duration=20.0 / scale)
        fields = {k: scatter_global(v, lay) for k, v in f.items()}
        return Workload(name, lay, h, 0.9, 1.0, 1.0, steps or 400, "vacuum", fields, {})
    if name in ("hybrid_1024", "local_1024"):
        gx, gy = 1024 // scale, 256 // scale
        ng = 64 // scale
        p = 64 // scale if scale > 1 else 64
        if name == "hybrid_1024":
            lay = hybrid_layout((gx, gy, gy), (4, 1, 1), ng, p)
        else:
            lay = local_layout((gx, gy, gy), (16, 4, 4), ng, p)
        f = laser_fields((gx, gy, gy), h, 1.0, wavelength=16.0 / scale,
                         waist=32.0 / scale, duration=20.0 / scale)
        fields = {k: scatter_global(v, lay) for k, v in f.items()}
        return Workload(name, lay, h, 0.9, 1.0, 1.0, steps or 200, "vacuum", fields, {})
    if name == "uneven_300":
        if scale > 1:
            lay = independent_layout(seed=5, nboxes=max(300 // (scale ** 3), 6),
                                     sizes=(16, 20, 24, 30, 32), ngs=(2, 4, 6),
                                     min_interior=8)
        else:
            lay = independent_layout(seed=5)
        rng = np.random.default_rng(5_000_005)
        js = {k: [] for k in ("Jx", "Jy", "Jz")}
        for b in lay.boxes:
            j = band_limited_current(b.interior, rng, h)
            for k in js:
                js[k].append(j[k])
        fields = {k: zeros(lay) for k in COMPONENTS}
        src = {k: scatter_self(v, lay) for k, v in js.items()}
        src["rho"] = zeros(lay)
        return Workload(name, lay, h, 0.9, 1.0, 1.0, steps or 100, "rho", fields, src)
    raise KeyError(name)


WORKLOADS = ("plane_waves_32", "sources_128", "local_512", "hybrid_1024",
             "local_1024", "uneven_300")
