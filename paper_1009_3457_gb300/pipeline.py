"""M2L over a stream of host-resident problems with the transfers overlapped.

``HostStreamM2L`` wraps the library's ``fmm_host_stream_*`` pipeline: each
step copies its MEs in from host memory, runs ``fmm_m2l_levels`` and copies the
LEs back out, on three CUDA streams that the library owns (host-to-device
copies, translation, device-to-host copies) with ``depth`` device buffer sets,
so that step i's translation runs while step i+1's MEs arrive and step i-1's
LEs leave.  The ordering (events, buffer reuse) is the library's; this class
only marshals torch tensors and exposes the streams as torch streams so that a
caller can record events on them.
"""
from __future__ import annotations

import torch

from . import fmmgb


class HostStreamM2L:
    """Overlapped host -> device -> host M2L over levels lmin..lmax of one tree.

    Every step's inputs are either a list of host tensors ([4^l, p] complex64,
    one per level, radius-scaled as for ``fmm_m2l``; one copy per level) or one
    flat complex64 host tensor holding the levels back to back (``flat_size``,
    ``level_views``), which the library moves in a single copy
    (FMM_HOST_CONTIGUOUS); the outputs take the same form.
    Page-locked (pinned) tensors let the copies overlap.  ``run`` enqueues the
    steps and returns; call ``sync()`` (or wait on ``done``) before reading the
    outputs."""

    def __init__(self, tree, lmin: int, lmax: int, p: int, prec: int = fmmgb.FMM_FP32, depth: int = 2,
                 device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.lmin, self.p, self.prec, self.depth = lmin, p, prec, depth
        self.levels = list(range(lmin, lmax + 1))
        with torch.cuda.device(dev):
            self.hs = fmmgb.fmm_host_stream_create(tree, lmin, lmax, p, prec, depth)
        info = self.hs.info()
        self.h2d, self.comp, self.d2h = (torch.cuda.ExternalStream(info[k], device=dev)
                                         for k in ("h2d_stream", "compute_stream", "d2h_stream"))
        self.done = torch.cuda.Event()

    def flat_size(self) -> int:
        """Complex entries of all levels back to back."""
        return sum(4 ** l for l in self.levels) * self.p

    def level_views(self, flat):
        """[4^l, p] views of the levels in a flat tensor of ``flat_size()`` entries."""
        out, off = [], 0
        for l in self.levels:
            n = 4 ** l * self.p
            out.append(flat[off:off + n].view(4 ** l, self.p))
            off += n
        return out

    def _levels(self, x):
        """A flat tensor goes whole (one copy per direction); a list goes level by level."""
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.complex64 or x.numel() != self.flat_size():
                raise fmmgb.FmmError(fmmgb.FMM_EINVAL, f"expected a flat complex64 tensor of {self.flat_size()}")
            return x
        views = list(x)
        for v, l in zip(views, self.levels):
            if v.dtype != torch.complex64 or tuple(v.shape) != (4 ** l, self.p):
                raise fmmgb.FmmError(fmmgb.FMM_EINVAL, f"level {l}: expected complex64 [{4 ** l}, {self.p}]")
        return views

    def run(self, host_in, host_out):
        """host_in[i], host_out[i]: step i's host MEs and LEs (per-level lists, or flat tensors,
        both of the same form)."""
        for Mh, Lh in zip(host_in, host_out):
            self.hs.submit(self._levels(Mh), self._levels(Lh))
        self.done.record(self.d2h)

    def sync(self):
        """Wait for every submitted step; raises on a device-side error."""
        self.hs.sync()

    @property
    def steps(self) -> int:
        return int(self.hs.info()["steps"])
