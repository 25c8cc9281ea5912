"""One hybrid group spread over several ranks: the distributed FFT's data
movement (paper Sec. 2.4.1) with the spectrum kept in the transposed layout
(Sec. 2.6, the "optimized communication strategy").

The paper runs each group's FFT on a sub-communicator of MPI ranks: a 3D FFT
transforms the axes one after the other, and before an axis whose lines are
split across ranks the array is transposed so that every rank holds whole
lines of it (Sec. 2.4.1).  A library keeps the output in the input's layout
by transposing back at the end; the paper's optimized strategy skips that
last transposition, solves Maxwell's equations in the transposed Fourier
layout, and starts the inverse transform from there (Sec. 2.6).

Here, on R ranks of one group (a torch.distributed process group):

* real space: rank r holds the z planes [z_r, z_{r+1}) of the group box,
  every (y, x) (a slab along the last axis, like the paper's FFTW mode);
* after the x and y transforms (R2C along x), rank r has the half spectrum
  (|Z_r|, n1, n0/2 + 1) of its planes;
* ``forward`` transposes (one all-to-all for all components): rank r then
  holds the rows my in [y_r, y_{r+1}) for every mz, layout (n2, |Y_r|,
  n0/2 + 1) with mx fastest -- a contiguous sub-box of the group spectrum in
  which the rank transforms z, updates every mode (the update is pointwise in
  k, so the layout is free; a mode's wavenumbers come from its global
  indices, y offset y_r) and transforms z back;
* ``inverse`` transposes back to the z slabs for the inverse y, x
  transforms.

So a step moves the spectrum twice (one all-to-all each way) instead of the
four transpositions of an FFT that restores its input layout in both
directions.  The transfers land in buffers of the receiving rank (NCCL on
GPUs, gloo on CPUs), no remote memory is read in place.

The per-rank transforms and the update are supplied to ``GroupStep`` as
three callables; ``DeviceRank`` gives them on the GPU through libpsatd.so
(psatd_plan_distribute and the psatd_dist_* calls: the rank's x, y
transforms of its slab, its z transform + update + inverse z transform of
its rows, its inverse y, x transforms), and this module does the partition
and the exchange.  With one GPU per machine here, the multi-rank exchange is
exercised with gloo ranks on the CPU, and the device work of several ranks
with the exchange done by copies on one GPU; the path is unmeasured on
several GPUs.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Sequence, Tuple

import torch
import torch.distributed as dist


def slab_bounds(n: int, parts: int) -> List[Tuple[int, int]]:
    """Split [0, n) into `parts` contiguous ranges whose sizes differ by at
    most one (the larger ones first)."""
    if parts < 1 or n < parts:
        raise ValueError(f"cannot split {n} planes over {parts} ranks")
    q, r = divmod(n, parts)
    out, lo = [], 0
    for i in range(parts):
        hi = lo + q + (1 if i < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


class SlabTranspose:
    """Partition of one group box (n0, n1, n2) over `world` ranks and the two
    transpositions of its half spectrum (see the module docstring).
    Tensors are complex (or real with a trailing size-2 axis) and may carry
    leading batch axes (components); the last three axes are the layout."""

    def __init__(self, n: Sequence[int], world: int, rank: int, group=None):
        self.n0, self.n1, self.n2 = (int(v) for v in n)
        self.hx = self.n0 // 2 + 1
        self.world, self.rank, self.group = int(world), int(rank), group
        self.z = slab_bounds(self.n2, self.world)    # real-space planes per rank
        self.y = slab_bounds(self.n1, self.world)    # spectrum rows per rank after the transposition
        self.transpositions = 0

    @property
    def z_slab(self) -> Tuple[int, int]:
        return self.z[self.rank]

    @property
    def y_rows(self) -> Tuple[int, int]:
        return self.y[self.rank]

    def _exchange(self, send_blocks, recv_shapes, like):
        """all-to-all of per-destination blocks; returns per-source blocks."""
        flat = [b.reshape(-1) for b in send_blocks]
        send = torch.cat(flat) if flat else like.new_zeros(0)
        in_split = [f.numel() for f in flat]
        out_split = [int(torch.Size(s).numel()) for s in recv_shapes]
        recv = like.new_empty(sum(out_split))
        if self.world == 1:
            recv.copy_(send)
        else:
            dist.all_to_all_single(recv, send, out_split, in_split, group=self.group)
        self.transpositions += 1
        out, off = [], 0
        for s, c in zip(recv_shapes, out_split):
            out.append(recv[off:off + c].view(*s))
            off += c
        return out

    @staticmethod
    def _real(t):
        return torch.view_as_real(t) if t.is_complex() else t

    def forward(self, spec: torch.Tensor) -> torch.Tensor:
        """(..., |Z_r|, n1, hx) -> (..., n2, |Y_r|, hx): z slabs to y rows."""
        cplx = spec.is_complex()
        x = self._real(spec.contiguous())
        lead = x.shape[:-4] if cplx else x.shape[:-3]
        tail = (2,) if cplx else ()
        zr = self.z_slab[1] - self.z_slab[0]
        ax = x.dim() - len(tail) - 2          # the y axis
        send = [x.narrow(ax, lo, hi - lo).contiguous() for lo, hi in self.y]
        yr = self.y_rows[1] - self.y_rows[0]
        shapes = [tuple(lead) + (hi - lo, yr, self.hx) + tail for lo, hi in self.z]
        blocks = self._exchange(send, shapes, x)
        out = torch.cat(blocks, dim=ax - 1)
        assert out.shape[ax - 1] == self.n2 and zr == spec.shape[-3]
        return torch.view_as_complex(out) if cplx else out

    def inverse(self, spec: torch.Tensor) -> torch.Tensor:
        """(..., n2, |Y_r|, hx) -> (..., |Z_r|, n1, hx): y rows back to z slabs."""
        cplx = spec.is_complex()
        x = self._real(spec.contiguous())
        lead = x.shape[:-4] if cplx else x.shape[:-3]
        tail = (2,) if cplx else ()
        az = x.dim() - len(tail) - 3          # the z axis
        send = [x.narrow(az, lo, hi - lo).contiguous() for lo, hi in self.z]
        zr = self.z_slab[1] - self.z_slab[0]
        shapes = [tuple(lead) + (zr, hi - lo, self.hx) + tail for lo, hi in self.y]
        blocks = self._exchange(send, shapes, x)
        out = torch.cat(blocks, dim=az + 1)
        return torch.view_as_complex(out) if cplx else out


class GroupStep:
    """One PSATD step of a group box distributed over the ranks of a process
    group, with the spectrum solved in the transposed layout.

    xy_forward(slab) -> spectrum: the x (R2C) and y transforms of every
        component of the rank's real slab (C, |Z_r|, n1, n0) into
        (C, |Z_r|, n1, hx);
    z_update(spec, y_lo) -> spec: z transform, per-mode update, inverse z
        transform of the rank's rows (C, n2, |Y_r|, hx), y_lo the global
        index of its first row;
    yx_inverse(spec) -> slab: the inverse y and x (C2R, 1/N) transforms.
    The three are the per-rank device work; this class does the two
    transpositions between them."""

    def __init__(self, n: Sequence[int], world: int, rank: int, xy_forward: Callable, z_update: Callable,
                 yx_inverse: Callable, group=None):
        self.t = SlabTranspose(n, world, rank, group)
        self.xy_forward, self.z_update, self.yx_inverse = xy_forward, z_update, yx_inverse

    def __call__(self, slab: torch.Tensor) -> torch.Tensor:
        spec = self.xy_forward(slab)
        rows = self.t.forward(spec)
        rows = self.z_update(rows, self.t.y_rows[0])
        return self.yx_inverse(self.t.inverse(rows))


def split_components(fields: Dict[str, torch.Tensor], names: Sequence[str], t: SlabTranspose) -> torch.Tensor:
    """The rank's z slab of every named component of full group arrays
    (n2, n1, n0), stacked: (C, |Z_r|, n1, n0)."""
    lo, hi = t.z_slab
    return torch.stack([fields[k][lo:hi] for k in names])


class DeviceRank:
    """The device work of rank `rank` of `world` for a ``GroupStep``: `plan`
    (a ``solver.Plan`` of the group box alone) distributed with
    psatd_plan_distribute.  Tensors live on the plan's device, components
    stacked along the first axis in slot order (Ex, Ey, Ez, Bx, By, Bz, then
    Jx, Jy, Jz with a current, or rho, Jx, Jy, Jz with a charge):
      xy_forward(slab (F, |Z_r|, n1, n0)) -> (F, |Z_r|, n1, n0/2 + 1) complex;
      z_update(rows (F, n2, |Y_r|, n0/2 + 1), y_lo) -> rows, in place;
      yx_inverse(spec (F, |Z_r|, n1, n0/2 + 1)) -> (F_out, |Z_r|, n1, n0): the
        output slots (E, B, and rho' with a charge) in a copy of the last
        slab given to xy_forward, whose x-face guard cells are left as they
        were.  `spec` is overwritten."""

    def __init__(self, plan, world: int, rank: int):
        from . import _abi as A
        self.A = A
        self.plan = plan
        A.psatd_plan_distribute(plan.handle, int(world), int(rank))
        self.z0, self.z1, self.y0, self.y1 = A.psatd_dist_bounds(plan.handle)
        self.n0, self.n1, self.n2 = (int(v) for v in plan.layout.boxes[0].n)
        self.hx = self.n0 // 2 + 1
        self.nf = {"vacuum": 6, "J": 9, "rho": 10}[plan.sources]
        self.nout = 7 if plan.sources == "rho" else 6
        self._last = None

    def _structs(self, slab):
        A = self.A
        es = slab.element_size() * slab.stride(0)
        ptr = [slab.data_ptr() + i * es for i in range(slab.shape[0])]
        f = A.psatd_fields()
        for a in range(3):
            f.E[a] = ptr[a]
            f.B[a] = ptr[3 + a]
        src = None
        if self.plan.sources != "vacuum":
            src = A.psatd_sources()
            j0 = 6 if self.plan.sources == "J" else 7
            for a in range(3):
                src.J[a] = ptr[j0 + a] if j0 + a < len(ptr) else None
            src.rho = ptr[6] if self.plan.sources == "rho" else None
        return f, src

    def _stream(self):
        import torch
        return torch.cuda.current_stream().cuda_stream

    def xy_forward(self, slab):
        import torch
        slab = slab.contiguous()
        if slab.shape != (self.nf, self.z1 - self.z0, self.n1, self.n0):
            raise ValueError(f"slab shape {tuple(slab.shape)}")
        cdt = torch.complex64 if slab.dtype == torch.float32 else torch.complex128
        spec = torch.empty((self.nf, self.z1 - self.z0, self.n1, self.hx), dtype=cdt, device=slab.device)
        f, src = self._structs(slab)
        self.A.psatd_dist_forward_xy(self.plan.handle, f, src, spec.data_ptr(), self._stream())
        self._last = slab
        return spec

    def z_update(self, rows, y_lo):
        if int(y_lo) != self.y0 or not rows.is_contiguous():
            raise ValueError("rows of another rank, or not contiguous")
        if rows.shape != (self.nf, self.n2, self.y1 - self.y0, self.hx):
            raise ValueError(f"rows shape {tuple(rows.shape)}")
        self.A.psatd_dist_z_update(self.plan.handle, rows.data_ptr(), self._stream())
        return rows

    def yx_inverse(self, spec):
        spec = spec.contiguous()
        out = self._last.clone()
        f, src = self._structs(out)
        self.A.psatd_dist_inverse_yx(self.plan.handle, spec.data_ptr(), f, src, self._stream())
        return out[:self.nout]
