"""Convenience layer over the C ABI: builds a plan description from a box
layout, and moves per-box numpy arrays in and out of the plan's contiguous
device buffers.  PyTorch provides device memory and the current stream;
all arithmetic of the push runs in libpsatd.so.
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional

import numpy as np

from . import _abi as A

_DECOMP = {"global": A.PSATD_DECOMP_GLOBAL, "local": A.PSATD_DECOMP_LOCAL,
           "hybrid": A.PSATD_DECOMP_HYBRID, "independent": A.PSATD_DECOMP_INDEPENDENT}
COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


def make_desc(layout, h, dt, c=1.0, eps0=1.0, precision=32, sources="vacuum", no_graph=False,
              generic=False, pencil=False, plane=False, j_constant=False, nodal=False, eager_exchange=False,
              pml=None, tuning=None):
    """psatd_plan_desc for an ``inputs.Layout``; the returned object keeps the
    box array alive (attribute ``_boxes``).  pml: absorbing layers,
    dict(width=(wx, wy, wz), sigma_max=(sx, sy, sz), order=m), or None.
    tuning: {knob name (see _abi.TUNE_KNOBS): value} launch parameters."""
    nb = len(layout.boxes)
    arr = (A.psatd_box * nb)()
    for i, b in enumerate(layout.boxes):
        arr[i].n[:] = list(b.n)
        arr[i].ng_lo[:] = list(b.ng_lo)
        arr[i].ng_hi[:] = list(b.ng_hi)
        arr[i].origin[:] = list(b.origin)
        arr[i].order_p = int(b.p)
    d = A.psatd_plan_desc()
    d.global_n[:] = list(layout.global_n)
    d.periodic[:] = list(layout.periodic)
    d.dx[:] = list(h)
    d.dt, d.c, d.eps0 = float(dt), float(c), float(eps0)
    d.precision = int(precision)
    d.decomp = _DECOMP[layout.kind]
    d.num_boxes = nb
    d.boxes = ctypes.cast(arr, ctypes.POINTER(A.psatd_box))
    flags = {"vacuum": A.PSATD_VACUUM, "J": 0, "rho": A.PSATD_RHO_CONTINUITY}[sources]
    if no_graph:
        flags |= A.PSATD_NO_GRAPH
    if generic:
        flags |= A.PSATD_GENERIC_KERNELS
    if pencil:
        flags |= A.PSATD_PENCIL_KERNELS
    if plane:
        flags |= A.PSATD_PLANE_KERNELS
    if j_constant:
        flags |= A.PSATD_J_CONSTANT
    if nodal:
        flags |= A.PSATD_NODAL
    if eager_exchange:
        flags |= A.PSATD_EAGER_EXCHANGE
    d.flags = flags
    d._boxes = arr
    if pml is not None:
        pm = A.psatd_pml()
        pm.width[:] = [int(v) for v in pml["width"]]
        pm.sigma_max[:] = [float(v) for v in pml["sigma_max"]]
        pm.order = int(pml["order"])
        d.pml = ctypes.pointer(pm)
        d._pml = pm
    if tuning:
        pairs = [v for k, x in sorted(tuning.items()) for v in (A.TUNE_KNOBS[k], int(x))] + [0, 0]
        arr_t = (ctypes.c_int32 * len(pairs))(*pairs)
        d.tuning = ctypes.cast(arr_t, ctypes.POINTER(ctypes.c_int32))
        d._tuning = arr_t
    return d


class Plan:
    """A PSATD plan on the current CUDA device."""

    def __init__(self, layout, h, dt, c=1.0, eps0=1.0, precision=32, sources="vacuum",
                 stream=None, no_graph=False, generic=False, pencil=False, plane=False, j_constant=False,
                 nodal=False, eager_exchange=False, pml=None, tuning=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.torch = torch
        self.layout = layout
        self.precision = precision
        self.sources = sources
        self.dtype = torch.float32 if precision == 32 else torch.float64
        self.cdtype = torch.complex64 if precision == 32 else torch.complex128
        self.np_dtype = np.float32 if precision == 32 else np.float64
        self.desc = make_desc(layout, h, dt, c, eps0, precision, sources, no_graph, generic, pencil, plane,
                              j_constant, nodal, eager_exchange, pml, tuning)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = A.psatd_plan_create(self.desc, self.stream.cuda_stream)
        self.offsets = [A.psatd_plan_layout(self.handle, i) for i in range(len(layout.boxes))]
        self.spec_offsets = [A.psatd_plan_spectrum_layout(self.handle, i)
                             for i in range(len(layout.boxes))]
        fb, wb = A.psatd_plan_memory(self.handle)
        self.field_elems = fb // (4 if precision == 32 else 8)
        self.workspace_bytes = wb
        self.fast_boxes = A.psatd_plan_fast_boxes(self.handle)
        self.pencil_boxes = A.psatd_plan_pencil_boxes(self.handle)
        self.deferred_exchange = bool(A.psatd_plan_deferred_exchange(self.handle))
        last = self.spec_offsets[-1]
        self.spec_elems = last[0] + last[1] + 64

    def close(self):
        if getattr(self, "handle", None):
            A.psatd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers -------------------------------------------------------------
    def empty(self):
        return self.torch.zeros(self.field_elems, dtype=self.dtype, device="cuda")

    def pack(self, arrays: List[np.ndarray]):
        host = np.zeros(self.field_elems, dtype=self.np_dtype)
        for (off, n), a in zip(self.offsets, arrays):
            host[off:off + n] = np.asarray(a, dtype=self.np_dtype).ravel()
        return self.torch.from_numpy(host).to("cuda")

    def unpack(self, t) -> List[np.ndarray]:
        host = t.detach().cpu().numpy().astype(np.float64)
        return [host[off:off + n].reshape(b.shape).copy()
                for (off, n), b in zip(self.offsets, self.layout.boxes)]

    def pack_separable(self, factors):
        """Device buffer from per-box separable factors (see
        ``inputs.laser_box_factors``); None gives zeros."""
        t = self.empty()
        if factors is None:
            return t
        torch = self.torch
        for (off, n), (fz, fy, fx, d) in zip(self.offsets, factors):
            z = torch.from_numpy(np.ascontiguousarray(fz)).cuda()
            y = torch.from_numpy(np.ascontiguousarray(fy)).cuda()
            x = torch.from_numpy(np.ascontiguousarray(fx)).cuda()
            v = (z.view(-1, 1, 1) * y.view(1, -1, 1) * x.view(1, 1, -1)) / d
            t[off:off + n] = v.reshape(-1).to(self.dtype)
        return t

    def pack_fields(self, d: Dict[str, List[np.ndarray]]):
        return {k: self.pack(v) for k, v in d.items()}

    def unpack_fields(self, d):
        return {k: self.unpack(v) for k, v in d.items()}

    # -- ABI structs ---------------------------------------------------------
    @staticmethod
    def fields_struct(f) -> A.psatd_fields:
        s = A.psatd_fields()
        s.E[:] = [f["Ex"].data_ptr(), f["Ey"].data_ptr(), f["Ez"].data_ptr()]
        s.B[:] = [f["Bx"].data_ptr(), f["By"].data_ptr(), f["Bz"].data_ptr()]
        return s

    @staticmethod
    def sources_struct(s) -> Optional[A.psatd_sources]:
        if not s:
            return None
        r = A.psatd_sources()
        r.J[:] = [s["Jx"].data_ptr(), s["Jy"].data_ptr(), s["Jz"].data_ptr()]
        r.rho = s["rho"].data_ptr() if s.get("rho") is not None else None
        return r

    # -- entry points ----------------------------------------------------------
    def push(self, fields, sources=None, nsteps=1):
        A.psatd_push(self.handle, self.fields_struct(fields), self.sources_struct(sources),
                     int(nsteps), self.stream.cuda_stream)

    def push_host(self, host_in, host_out=None, sources=None, nsteps=1):
        """psatd_push_host: fields in host tensors (dict component -> CPU
        tensor of field_elems, page-locked for speed); results in host_out
        (default: in place)."""
        host_out = host_in if host_out is None else host_out
        A.psatd_push_host(self.handle, self.fields_struct(host_in), self.fields_struct(host_out),
                          self.sources_struct(sources), int(nsteps), self.stream.cuda_stream)

    def push_host_global(self, host_in, host_out=None, sources=None, nsteps=1):
        """psatd_push_host_global: fields as whole-domain host tensors (dict
        component -> CPU tensor of global_n[0]*global_n[1]*global_n[2],
        x fastest); results in host_out (default: in place)."""
        host_out = host_in if host_out is None else host_out
        A.psatd_push_host_global(self.handle, self.fields_struct(host_in), self.fields_struct(host_out),
                                 self.sources_struct(sources), int(nsteps), self.stream.cuda_stream)

    def guard_exchange(self, fields, sources=None):
        A.psatd_guard_exchange(self.handle, self.fields_struct(fields),
                               self.sources_struct(sources), self.stream.cuda_stream)

    def forward_fft(self, field):
        spec = self.torch.zeros(self.spec_elems, dtype=self.cdtype, device="cuda")
        A.psatd_forward_fft(self.handle, field.data_ptr(), spec.data_ptr(), self.stream.cuda_stream)
        return spec

    def inverse_fft(self, spec):
        out = self.empty()
        A.psatd_inverse_fft(self.handle, spec.data_ptr(), out.data_ptr(), self.stream.cuda_stream)
        return out

    def unpack_spectrum(self, spec) -> List[np.ndarray]:
        host = spec.detach().cpu().numpy().astype(np.complex128)
        out = []
        for (off, n), b in zip(self.spec_offsets, self.layout.boxes):
            out.append(host[off:off + n].reshape(b.n[2], b.n[1], b.n[0] // 2 + 1).copy())
        return out

    def sync(self):
        A.psatd_sync_status(self.handle)

    # the stored split parts of the absorbing layers (plan-owned device memory)
    PML_PARTS = ("Exy", "Eyz", "Ezx", "Bxy", "Byz", "Bzx")

    def pml_parts(self):
        """{name: tensor} views of the plan's stored split parts (same layout
        as a field buffer; zero-copy through __cuda_array_interface__)."""
        out = {}
        for q, name in enumerate(self.PML_PARTS):
            ptr = A.psatd_plan_pml_part(self.handle, q)
            out[name] = self.torch.as_tensor(_DeviceArray(ptr, self.field_elems, self.precision), device="cuda")
        return out

    def last_launch_count(self) -> int:
        return A.psatd_last_launch_count(self.handle)

    def tuning(self):
        """{knob name: value} of the knobs this plan's kernels use."""
        out = {}
        for name, k in A.TUNE_KNOBS.items():
            v = A.psatd_plan_tuning(self.handle, k)
            if v >= 0:
                out[name] = v
        return out


class _DeviceArray:
    """A device buffer owned by the library, exposed to torch without a copy."""

    def __init__(self, ptr, n, precision):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f4" if precision == 32 else "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class Coupling:
    """Dual-grid coupling of a plan's FFT boxes (G2) with a second
    decomposition G1 of the same domain (an ``inputs.Layout`` whose boxes may
    have any sizes and guard widths): ``to_fft`` fills every G2 cell from the
    G1 interiors, ``from_fft`` every G1 cell from the G2 interiors."""

    def __init__(self, plan, g1_layout):
        self.plan = plan
        self.g1 = g1_layout
        self.handle = A.psatd_coupling_create(plan.handle, g1_layout.boxes)
        self.offsets = [A.psatd_coupling_layout(self.handle, i) for i in range(len(g1_layout.boxes))]
        last = self.offsets[-1]
        self.elems = last[0] + last[1] + 64

    def close(self):
        if self.handle:
            A.psatd_coupling_destroy(self.handle)
            self.handle = None

    def empty(self):
        return self.plan.torch.zeros(self.elems, dtype=self.plan.dtype, device="cuda")

    def pack(self, arrays: List[np.ndarray]):
        t = self.empty()
        for (off, n), a in zip(self.offsets, arrays):
            t[off:off + n] = self.plan.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(
                device="cuda", dtype=self.plan.dtype)
        return t

    def unpack(self, t) -> List[np.ndarray]:
        h = t.detach().to("cpu", dtype=self.plan.torch.float64).numpy()
        return [h[off:off + n].reshape(b.shape).copy() for (off, n), b in zip(self.offsets, self.g1.boxes)]

    def _run(self, direction, g1: Dict, g2: Dict):
        keys = [k for k in g1 if k in g2]
        A.psatd_couple(self.handle, direction, [g1[k].data_ptr() for k in keys], [g2[k].data_ptr() for k in keys],
                       self.plan.stream.cuda_stream, self.plan.handle)

    def to_fft(self, g1: Dict, g2: Dict):
        self._run(A.PSATD_G1_TO_G2, g1, g2)

    def from_fft(self, g2: Dict, g1: Dict):
        self._run(A.PSATD_G2_TO_G1, g1, g2)
