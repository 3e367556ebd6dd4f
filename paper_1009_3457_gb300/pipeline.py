"""M2L over a stream of host-resident problems with the transfers overlapped.

``HostStreamM2L`` runs ``fmm_m2l_levels`` on a sequence of multipole sets that
live in (pinned) host memory and returns the local expansions to host memory.
Each step copies its MEs in, translates them and copies the LEs out; with
``depth`` device buffer sets and three CUDA streams (host-to-device copies,
translation, device-to-host copies), step i's translation runs while step i+1's
MEs are arriving and step i-1's LEs are leaving, so the link's two directions
and the SMs work at the same time.  The two halves of a buffer set are released
separately (CUDA events order the streams): a step's MEs may arrive as soon as
the translation that last read that ME buffer is done, while its translation
waits until the LEs last written to its LE buffer have been copied out.  So the
copy in of step i+1 overlaps the copy out of step i-1, and with two buffer sets
a step costs the longest of the translation and the two concurrent copies, not
their sum.
"""
from __future__ import annotations

import torch

from . import fmmgb


class HostStreamM2L:
    """Overlapped host -> device -> host M2L over levels lmin..lmax of one tree.

    Every step's inputs are either a list of pinned host tensors ([4^l, p] complex64,
    one per level, radius-scaled as for ``fmm_m2l``) or one flat pinned complex64
    tensor holding the levels back to back (``flat_size``, ``level_views``), which
    moves in a single copy; the outputs take the same form.  ``run`` enqueues the
    steps and returns; call ``torch.cuda.synchronize()`` (or wait on ``done``)
    before reading the outputs."""

    def __init__(self, tree, lmin: int, lmax: int, p: int, prec: int = fmmgb.FMM_FP32, depth: int = 2,
                 device=None):
        if depth < 1:
            raise ValueError("depth must be at least 1")
        self.tree, self.lmin, self.p, self.prec, self.depth = tree, lmin, p, prec, depth
        self.levels = list(range(lmin, lmax + 1))
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.h2d, self.comp, self.d2h = (torch.cuda.Stream(device=dev) for _ in range(3))
        self.Mflat = [torch.empty(self.flat_size(), dtype=torch.complex64, device=dev) for _ in range(depth)]
        self.Lflat = [torch.empty_like(m) for m in self.Mflat]
        self.M = [self.level_views(m) for m in self.Mflat]
        self.L = [self.level_views(m) for m in self.Lflat]
        self.arrived = [torch.cuda.Event() for _ in range(depth)]
        self.translated = [torch.cuda.Event() for _ in range(depth)]
        self.returned = [torch.cuda.Event() for _ in range(depth)]
        self.done = torch.cuda.Event()
        self.steps = 0

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

    @staticmethod
    def _copy(dst_flat, dst_views, src):
        if isinstance(src, torch.Tensor):
            dst_flat.copy_(src, non_blocking=True)
        else:
            for d, x in zip(dst_views, src):
                d.copy_(x, non_blocking=True)

    def run(self, host_in, host_out):
        """host_in[i], host_out[i]: step i's pinned host MEs and LEs (per-level lists or flat tensors)."""
        for Mh, Lh in zip(host_in, host_out):
            b = self.steps % self.depth
            if self.steps >= self.depth:
                # set b's MEs were last read by the translation of step steps - depth, its
                # LEs last copied out by that step's copy out
                self.h2d.wait_event(self.translated[b])
                self.comp.wait_event(self.returned[b])
            with torch.cuda.stream(self.h2d):
                self._copy(self.Mflat[b], self.M[b], Mh)
                self.arrived[b].record(self.h2d)
            self.comp.wait_event(self.arrived[b])
            fmmgb.fmm_m2l_levels(self.tree, self.lmin, self.p, self.M[b], self.L[b], prec=self.prec,
                                 stream=self.comp)
            self.translated[b].record(self.comp)
            self.d2h.wait_event(self.translated[b])
            with torch.cuda.stream(self.d2h):
                if isinstance(Lh, torch.Tensor):
                    Lh.copy_(self.Lflat[b], non_blocking=True)
                else:
                    for dst, src in zip(Lh, self.L[b]):
                        dst.copy_(src, non_blocking=True)
                self.returned[b].record(self.d2h)
            self.steps += 1
        self.done.record(self.d2h)
