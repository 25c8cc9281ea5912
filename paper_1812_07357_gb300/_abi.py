"""ctypes binding of include/psatd.h: argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; a missing or unbuilt library raises immediately (there
is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_int32, c_int64,
                    c_size_t, c_uint32, c_void_p)

from . import build as _build

PSATD_OK = 0
PSATD_ERR_INVALID_ARG = 1
PSATD_ERR_UNSUPPORTED_SIZE = 2
PSATD_ERR_UNSUPPORTED_ORDER = 3
PSATD_ERR_OUT_OF_MEMORY = 4
PSATD_ERR_CUDA = 5
PSATD_ERR_TIMEOUT = 6
PSATD_ERR_STATE = 7

PSATD_DECOMP_GLOBAL = 0
PSATD_DECOMP_LOCAL = 1
PSATD_DECOMP_HYBRID = 2
PSATD_DECOMP_INDEPENDENT = 3

PSATD_VACUUM = 0x1
PSATD_RHO_CONTINUITY = 0x2
PSATD_NO_GRAPH = 0x8
PSATD_GENERIC_KERNELS = 0x10
PSATD_PENCIL_KERNELS = 0x20
PSATD_J_CONSTANT = 0x4
PSATD_PLANE_KERNELS = 0x40
PSATD_NODAL = 0x80
PSATD_EAGER_EXCHANGE = 0x100


class psatd_box(Structure):
    _fields_ = [("n", c_int32 * 3), ("ng_lo", c_int32 * 3), ("ng_hi", c_int32 * 3),
                ("origin", c_int64 * 3), ("order_p", c_int32)]


class psatd_pml(Structure):
    _fields_ = [("width", c_int32 * 3), ("sigma_max", c_double * 3), ("order", c_int32)]


class psatd_plan_desc(Structure):
    _fields_ = [("global_n", c_int32 * 3), ("periodic", c_int32 * 3), ("dx", c_double * 3),
                ("dt", c_double), ("c", c_double), ("eps0", c_double), ("precision", c_int32),
                ("decomp", c_int32), ("num_boxes", c_int32), ("boxes", POINTER(psatd_box)),
                ("flags", c_uint32), ("pml", POINTER(psatd_pml)), ("tuning", POINTER(c_int32))]


class psatd_fields(Structure):
    _fields_ = [("E", c_void_p * 3), ("B", c_void_p * 3)]


class psatd_sources(Structure):
    _fields_ = [("J", c_void_p * 3), ("rho", c_void_p)]


class psatd_copy_block(Structure):
    _fields_ = [("dst_box", c_int32), ("src_box", c_int32), ("dst_lo", c_int32 * 3),
                ("src_lo", c_int32 * 3), ("ext", c_int32 * 3)]


class PsatdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


_SIGS = {
    "psatd_plan_validate": (c_int32, [POINTER(psatd_plan_desc), c_char_p, c_size_t]),
    "psatd_exchange_blocks": (c_int32, [POINTER(psatd_plan_desc), POINTER(psatd_copy_block),
                                        c_int64, POINTER(c_int64)]),
    "psatd_plan_create": (c_int32, [POINTER(psatd_plan_desc), c_void_p, POINTER(c_void_p)]),
    "psatd_plan_destroy": (c_int32, [c_void_p]),
    "psatd_plan_layout": (c_int32, [c_void_p, c_int32, POINTER(c_int64), POINTER(c_int64)]),
    "psatd_plan_memory": (c_int32, [c_void_p, POINTER(c_size_t), POINTER(c_size_t)]),
    "psatd_guard_exchange": (c_int32, [c_void_p, POINTER(psatd_fields), POINTER(psatd_sources),
                                       c_void_p]),
    "psatd_push": (c_int32, [c_void_p, POINTER(psatd_fields), POINTER(psatd_sources), c_int32,
                             c_void_p]),
    "psatd_forward_fft": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "psatd_inverse_fft": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "psatd_plan_spectrum_layout": (c_int32, [c_void_p, c_int32, POINTER(c_int64),
                                             POINTER(c_int64)]),
    "psatd_plan_distribute": (c_int32, [c_void_p, c_int32, c_int32]),
    "psatd_dist_bounds": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32),
                                    POINTER(c_int32)]),
    "psatd_dist_forward_xy": (c_int32, [c_void_p, POINTER(psatd_fields), POINTER(psatd_sources), c_void_p,
                                        c_void_p]),
    "psatd_dist_z_update": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "psatd_dist_inverse_yx": (c_int32, [c_void_p, c_void_p, POINTER(psatd_fields), POINTER(psatd_sources),
                                        c_void_p]),
    "psatd_sync_status": (c_int32, [c_void_p]),
    "psatd_status_string": (c_char_p, [c_int32]),
    "psatd_last_error": (c_char_p, [c_void_p]),
    "psatd_last_launch_count": (c_int64, [c_void_p]),
    "psatd_plan_set_timing": (c_int32, [c_void_p, c_int32]),
    "psatd_plan_tune": (c_int32, [c_void_p, c_int32, c_int32]),
    "psatd_push_host": (c_int32, [c_void_p, POINTER(psatd_fields), POINTER(psatd_fields), POINTER(psatd_sources),
                                  c_int32, c_void_p]),
    "psatd_push_host_global": (c_int32, [c_void_p, POINTER(psatd_fields), POINTER(psatd_fields),
                                         POINTER(psatd_sources), c_int32, c_void_p]),
    "psatd_plan_pml_part": (c_int32, [c_void_p, c_int32, POINTER(c_void_p)]),
    "psatd_plan_tuning": (c_int32, [c_void_p, c_int32]),
    "psatd_plan_kernel_times": (c_int32, [c_void_p, POINTER(c_double), POINTER(c_int64), c_int32]),
    "psatd_plan_fast_boxes": (c_int32, [c_void_p]),
    "psatd_plan_pencil_boxes": (c_int32, [c_void_p]),
    "psatd_plan_deferred_exchange": (c_int32, [c_void_p]),
    "psatd_push_box_static": (c_int32, [POINTER(c_int32), c_int32, POINTER(c_double), c_double,
                                        c_double, POINTER(psatd_fields), c_int32, c_void_p]),
    "psatd_plane_gather": (c_int32, [POINTER(psatd_plan_desc), c_int32, c_int32, POINTER(c_int32), POINTER(c_int64),
                                     POINTER(c_int32)]),
    "psatd_coupling_blocks": (c_int32, [POINTER(psatd_plan_desc), c_int32, POINTER(psatd_box), c_int32,
                                        POINTER(psatd_copy_block), c_int64, POINTER(c_int64)]),
    "psatd_coupling_create": (c_int32, [c_void_p, c_int32, POINTER(psatd_box), POINTER(c_void_p)]),
    "psatd_coupling_destroy": (c_int32, [c_void_p]),
    "psatd_coupling_layout": (c_int32, [c_void_p, c_int32, POINTER(c_int64), POINTER(c_int64)]),
    "psatd_couple": (c_int32, [c_void_p, c_int32, POINTER(c_void_p), POINTER(c_void_p), c_int32, c_void_p]),
}

PSATD_G1_TO_G2 = 0
PSATD_G2_TO_G1 = 1

PSATD_STATIC_SCRATCH_BYTES = 64 << 20

PSATD_KERNEL_KINDS = 6
KERNEL_NAMES = ("fwd_xy", "col_fwd", "z_update", "col_inv", "inv_yx", "exchange")

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libpsatd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_1812_07357_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def status_name(s: int) -> str:
    try:
        return load().psatd_status_string(s).decode()
    except Exception:  # library unavailable while formatting an error
        return f"status {s}"


def _check(st, plan=None):
    if st != PSATD_OK:
        raise PsatdError(st, psatd_last_error(plan))


# --- one wrapper per entry point (same names) ------------------------------

def psatd_plan_validate(desc: psatd_plan_desc):
    buf = ctypes.create_string_buffer(512)
    st = load().psatd_plan_validate(ctypes.byref(desc), buf, 512)
    return st, buf.value.decode()


def psatd_exchange_blocks(desc: psatd_plan_desc):
    n = c_int64(0)
    _check(load().psatd_exchange_blocks(ctypes.byref(desc), None, 0, ctypes.byref(n)))
    arr = (psatd_copy_block * max(n.value, 1))()
    _check(load().psatd_exchange_blocks(ctypes.byref(desc), arr, n.value, ctypes.byref(n)))
    return [arr[i] for i in range(n.value)]


def _box_array(boxes):
    arr = (psatd_box * max(len(boxes), 1))()
    for i, b in enumerate(boxes):
        arr[i].n[:] = list(b.n)
        arr[i].ng_lo[:] = list(b.ng_lo)
        arr[i].ng_hi[:] = list(b.ng_hi)
        arr[i].origin[:] = list(b.origin)
        arr[i].order_p = int(b.p)
    return arr


def psatd_plane_gather(desc: psatd_plan_desc, box: int, z: int):
    """Host-only: (src_box, src_cell, is_grid) of plane z of `box` under the
    deferred guard exchange; the arrays have shape (n1, n0)."""
    import numpy as np
    if 0 <= box < desc.num_boxes:
        b = desc.boxes[box]
        n0, n1 = int(b.n[0]), int(b.n[1])
    else:
        n0 = n1 = 1          # the call reports the bad index without writing
    sb = np.empty(n0 * n1, dtype=np.int32)
    sc = np.empty(n0 * n1, dtype=np.int64)
    g = c_int32(0)
    _check(load().psatd_plane_gather(ctypes.byref(desc), box, z, sb.ctypes.data_as(POINTER(c_int32)),
                                     sc.ctypes.data_as(POINTER(c_int64)), ctypes.byref(g)))
    return sb.reshape(n1, n0), sc.reshape(n1, n0), bool(g.value)


def psatd_coupling_blocks(desc: psatd_plan_desc, g1_boxes, direction: int):
    """Host-only copy blocks of a dual-grid coupling (G1 boxes: objects with
    n, ng_lo, ng_hi, origin, p)."""
    arr = _box_array(g1_boxes)
    n = c_int64(0)
    _check(load().psatd_coupling_blocks(ctypes.byref(desc), len(g1_boxes), arr, direction, None, 0,
                                        ctypes.byref(n)))
    out = (psatd_copy_block * max(n.value, 1))()
    _check(load().psatd_coupling_blocks(ctypes.byref(desc), len(g1_boxes), arr, direction, out, n.value,
                                        ctypes.byref(n)))
    return [out[i] for i in range(n.value)]


def psatd_coupling_create(plan: int, g1_boxes) -> int:
    arr = _box_array(g1_boxes)
    out = c_void_p()
    _check(load().psatd_coupling_create(c_void_p(plan), len(g1_boxes), arr, ctypes.byref(out)), plan)
    return out.value


def psatd_coupling_destroy(coupling: int):
    _check(load().psatd_coupling_destroy(c_void_p(coupling)))


def psatd_coupling_layout(coupling: int, box: int):
    off, n = c_int64(), c_int64()
    _check(load().psatd_coupling_layout(c_void_p(coupling), box, ctypes.byref(off), ctypes.byref(n)))
    return off.value, n.value


def psatd_couple(coupling: int, direction: int, g1_ptrs, g2_ptrs, stream: int, plan: int = None):
    n = len(g1_ptrs)
    a1 = (c_void_p * n)(*g1_ptrs)
    a2 = (c_void_p * n)(*g2_ptrs)
    _check(load().psatd_couple(c_void_p(coupling), direction, a1, a2, n, c_void_p(stream)), plan)


def psatd_plan_create(desc: psatd_plan_desc, stream: int = 0) -> int:
    out = c_void_p()
    _check(load().psatd_plan_create(ctypes.byref(desc), c_void_p(stream), ctypes.byref(out)))
    return out.value


def psatd_plan_destroy(plan: int):
    _check(load().psatd_plan_destroy(c_void_p(plan)))


def psatd_plan_layout(plan: int, box: int):
    off, n = c_int64(), c_int64()
    _check(load().psatd_plan_layout(c_void_p(plan), box, ctypes.byref(off), ctypes.byref(n)), plan)
    return off.value, n.value


def psatd_plan_spectrum_layout(plan: int, box: int):
    off, n = c_int64(), c_int64()
    _check(load().psatd_plan_spectrum_layout(c_void_p(plan), box, ctypes.byref(off),
                                             ctypes.byref(n)), plan)
    return off.value, n.value


def psatd_plan_memory(plan: int):
    f, w = c_size_t(), c_size_t()
    _check(load().psatd_plan_memory(c_void_p(plan), ctypes.byref(f), ctypes.byref(w)), plan)
    return f.value, w.value


def psatd_guard_exchange(plan: int, fields: psatd_fields, src: psatd_sources | None,
                         stream: int = 0):
    _check(load().psatd_guard_exchange(c_void_p(plan), ctypes.byref(fields),
                                       ctypes.byref(src) if src is not None else None,
                                       c_void_p(stream)), plan)


def psatd_push(plan: int, fields: psatd_fields, src: psatd_sources | None, nsteps: int,
               stream: int = 0):
    _check(load().psatd_push(c_void_p(plan), ctypes.byref(fields),
                             ctypes.byref(src) if src is not None else None, nsteps,
                             c_void_p(stream)), plan)


def psatd_forward_fft(plan: int, field: int, spectrum: int, stream: int = 0):
    _check(load().psatd_forward_fft(c_void_p(plan), c_void_p(field), c_void_p(spectrum),
                                    c_void_p(stream)), plan)


def psatd_inverse_fft(plan: int, spectrum: int, field: int, stream: int = 0):
    _check(load().psatd_inverse_fft(c_void_p(plan), c_void_p(spectrum), c_void_p(field),
                                    c_void_p(stream)), plan)


def psatd_plan_distribute(plan: int, world: int, rank: int):
    _check(load().psatd_plan_distribute(c_void_p(plan), world, rank), plan)


def psatd_dist_bounds(plan: int):
    """(z0, z1, y0, y1): the rank's z slab and spectrum rows."""
    v = [c_int32() for _ in range(4)]
    _check(load().psatd_dist_bounds(c_void_p(plan), *(ctypes.byref(x) for x in v)), plan)
    return tuple(x.value for x in v)


def psatd_dist_forward_xy(plan: int, slab: psatd_fields, src: psatd_sources | None, slab_spectrum: int,
                          stream: int = 0):
    _check(load().psatd_dist_forward_xy(c_void_p(plan), ctypes.byref(slab),
                                        ctypes.byref(src) if src is not None else None, c_void_p(slab_spectrum),
                                        c_void_p(stream)), plan)


def psatd_dist_z_update(plan: int, rows: int, stream: int = 0):
    _check(load().psatd_dist_z_update(c_void_p(plan), c_void_p(rows), c_void_p(stream)), plan)


def psatd_dist_inverse_yx(plan: int, slab_spectrum: int, slab: psatd_fields, src: psatd_sources | None,
                          stream: int = 0):
    _check(load().psatd_dist_inverse_yx(c_void_p(plan), c_void_p(slab_spectrum), ctypes.byref(slab),
                                        ctypes.byref(src) if src is not None else None, c_void_p(stream)), plan)


def psatd_sync_status(plan: int):
    _check(load().psatd_sync_status(c_void_p(plan)), plan)


def psatd_status_string(s: int) -> str:
    return load().psatd_status_string(s).decode()


def psatd_last_error(plan: int | None = None) -> str:
    return load().psatd_last_error(c_void_p(plan) if plan else None).decode()


def psatd_last_launch_count(plan: int) -> int:
    return int(load().psatd_last_launch_count(c_void_p(plan)))


def psatd_plan_set_timing(plan: int, enable: bool):
    _check(load().psatd_plan_set_timing(c_void_p(plan), 1 if enable else 0), plan)


PSATD_TUNE_Z_PREFETCH = 1
PSATD_TUNE_PENCIL_ROWS_KB = 2
PSATD_TUNE_Z_TILE = 3
PSATD_TUNE_HOST_COPY = 4
PSATD_TUNE_PENCIL_REG_Z = 5
PSATD_TUNE_Z_ONE_LAUNCH = 6
PSATD_TUNE_REG_PLANES = 7
TUNE_KNOBS = {"z_prefetch": PSATD_TUNE_Z_PREFETCH, "pencil_rows_kb": PSATD_TUNE_PENCIL_ROWS_KB,
              "z_tile": PSATD_TUNE_Z_TILE, "host_copy": PSATD_TUNE_HOST_COPY,
              "pencil_reg_z": PSATD_TUNE_PENCIL_REG_Z, "z_one_launch": PSATD_TUNE_Z_ONE_LAUNCH,
              "reg_planes": PSATD_TUNE_REG_PLANES}


def psatd_push_host(plan: int, fin: psatd_fields, fout: psatd_fields, sources, nsteps: int, stream: int = 0):
    _check(load().psatd_push_host(c_void_p(plan), ctypes.byref(fin), ctypes.byref(fout),
                                  ctypes.byref(sources) if sources is not None else None, int(nsteps),
                                  c_void_p(stream)), plan)


def psatd_push_host_global(plan: int, fin: psatd_fields, fout: psatd_fields, sources, nsteps: int,
                           stream: int = 0):
    _check(load().psatd_push_host_global(c_void_p(plan), ctypes.byref(fin), ctypes.byref(fout),
                                         ctypes.byref(sources) if sources is not None else None, int(nsteps),
                                         c_void_p(stream)), plan)


def psatd_plan_pml_part(plan: int, q: int) -> int:
    out = c_void_p()
    _check(load().psatd_plan_pml_part(c_void_p(plan), int(q), ctypes.byref(out)), plan)
    return out.value


def psatd_plan_tune(plan: int, knob: int, value: int):
    _check(load().psatd_plan_tune(c_void_p(plan), int(knob), int(value)), plan)


def psatd_plan_tuning(plan: int, knob: int) -> int:
    return int(load().psatd_plan_tuning(c_void_p(plan), int(knob)))


def psatd_plan_kernel_times(plan: int):
    ms = (c_double * PSATD_KERNEL_KINDS)()
    n = (c_int64 * PSATD_KERNEL_KINDS)()
    _check(load().psatd_plan_kernel_times(c_void_p(plan), ms, n, PSATD_KERNEL_KINDS), plan)
    return list(ms), list(n)


def psatd_push_box_static(n, order_p: int, dx, dt: float, c: float, fields: psatd_fields,
                          nsteps: int, stream: int = 0):
    """One periodic FP32 vacuum box, pushed without any device allocation
    (scratch lives in the library's static device array)."""
    nn = (c_int32 * 3)(*[int(v) for v in n])
    dd = (c_double * 3)(*[float(v) for v in dx])
    _check(load().psatd_push_box_static(nn, int(order_p), dd, float(dt), float(c),
                                        ctypes.byref(fields), int(nsteps), c_void_p(stream)))


def psatd_plan_fast_boxes(plan: int) -> int:
    return int(load().psatd_plan_fast_boxes(c_void_p(plan)))


def psatd_plan_pencil_boxes(plan: int) -> int:
    return int(load().psatd_plan_pencil_boxes(c_void_p(plan)))


def psatd_plan_deferred_exchange(plan: int) -> int:
    return int(load().psatd_plan_deferred_exchange(c_void_p(plan)))
