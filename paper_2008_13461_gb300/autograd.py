"""Differentiable broken-line fit and hit alignment (torch.autograd).

``DifferentiableFit`` keeps the n-tuplets of one pipeline run fixed and
refits them from given hit coordinates (Sec. 3.4); the gradient of any loss
of the track parameters and chi2 flows back to the coordinates through the
library's adjoint kernel (``pt_fit_tracks_grad``), and from there to
per-module alignment shifts and rotations through ``pt_align_hits_grad``.
This module only marshals arguments: every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import _lib as L


class _Fit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, z, owner):
        params, chi2 = owner._fit(x, y, z)
        ctx.owner = owner
        ctx.save_for_backward(x, y, z)
        return params, chi2

    @staticmethod
    def backward(ctx, gparams, gchi2):
        x, y, z = ctx.saved_tensors
        gx, gy, gz = ctx.owner._fit_grad(x, y, z, gparams, gchi2)
        return gx, gy, gz, None


class _Align(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, z, shift, rot, owner):
        out = owner._align(x, y, z, shift, rot)
        ctx.owner = owner
        ctx.save_for_backward(x, y, z, rot)
        return out

    @staticmethod
    def backward(ctx, gxo, gyo, gzo):
        x, y, z, rot = ctx.saved_tensors
        gx, gy, gz, gshift, grot = ctx.owner._align_grad(x, y, z, rot, gxo, gyo, gzo, ctx.needs_input_grad)
        return gx, gy, gz, gshift, grot, None


class DifferentiableFit:
    """The tracks of a finished pipeline run, refittable from moved hits.

    ``fit(x, y, z)`` returns (params[K, 5], chi2[K]) for the run's tracks, in
    the run's (deterministic) track order, differentiable in x, y, z.
    ``align(x, y, z, shift, rot)`` moves the hits by per-module shifts and
    small rotations about ``centres`` (float[n_modules, 3]), differentiable in
    all of them.  Hit coordinates are float32 tensors on the pipeline's
    device; the hits' modules and events stay those of the run.

    A refit writes into track arrays of its own (allocated here at the
    run's track capacity), so the run's ``Result.tracks`` keep the fit of
    the original hits.  The refit still shares the run's workspace, whose
    track counters it sets to the same values (the selection of tracks
    depends on the n-tuplets only).
    """

    def __init__(self, pipe, bufs, r, module, ev_off, centres: torch.Tensor | None = None):
        self.pipe, self.bufs = pipe, bufs
        self.r, self.module, self.ev_off = r, module, ev_off
        self.centres = None if centres is None else centres.to(pipe.device, torch.float32).contiguous()
        nk = max(1, int(bufs.capacity["tracks"]))
        d = pipe.device
        self.params = torch.empty(nk * 5, dtype=torch.float32, device=d)
        self.cov = torch.empty(nk * 15, dtype=torch.float32, device=d)
        self.chi2 = torch.empty(nk, dtype=torch.float32, device=d)
        self.ndf = torch.empty(nk, dtype=torch.int8, device=d)
        self.tuple = torch.empty(nk, dtype=torch.int32, device=d)

    def _tracks(self) -> L.Tracks:
        return L.Tracks(self.params.data_ptr(), self.cov.data_ptr(), self.chi2.data_ptr(), self.ndf.data_ptr(),
                        self.tuple.data_ptr())

    # -- fit
    def _hits(self, x, y, z):
        return self.pipe._hits(x, y, z, self.r, self.module, self.ev_off)

    def _stream(self):
        return torch.cuda.current_stream(self.pipe.device).cuda_stream

    def fit(self, x, y, z):
        return _Fit.apply(x, y, z, self)

    def _fit(self, x, y, z):
        x, y, z = (t.detach().contiguous() for t in (x, y, z))
        b = self.bufs
        cfg = self.pipe._cfg(b.capacity)
        h = self._hits(x, y, z)
        _, _, tuples, _ = b.structs()
        s = self._stream()
        L.fit_tracks(b.ws.data_ptr(), b.ws.numel(), h, cfg, tuples, self._tracks(), s)
        st, c = L.read_counts(b.ws.data_ptr(), b.ws.numel(), h, cfg, s)
        L.check(st, "refit")
        k = c.n_tracks
        return self.params[:k * 5].view(k, 5).clone(), self.chi2[:k].clone()

    def _fit_grad(self, x, y, z, gparams, gchi2):
        x, y, z = (t.detach().contiguous() for t in (x, y, z))
        b = self.bufs
        dev = x.device
        gp = (gparams if gparams is not None else torch.zeros(0, 5, device=dev)).to(torch.float32).contiguous()
        gc = None if gchi2 is None else gchi2.to(torch.float32).contiguous()
        gx, gy, gz = (torch.zeros_like(x) for _ in range(3))
        if gparams is None:
            k = int(gc.numel()) if gc is not None else 0
            gp = torch.zeros(k, 5, device=dev)
        _, _, tuples, _ = b.structs()
        L.fit_tracks_grad(b.ws.data_ptr(), b.ws.numel(), self._hits(x, y, z), self.pipe._cfg(b.capacity), tuples,
                          self._tracks(), gp.data_ptr(), None if gc is None else gc.data_ptr(), gx.data_ptr(),
                          gy.data_ptr(), gz.data_ptr(), self._stream())
        return gx, gy, gz

    # -- alignment
    def align(self, x, y, z, shift, rot):
        return _Align.apply(x, y, z, shift, rot, self)

    def _align(self, x, y, z, shift, rot):
        if self.centres is None:
            raise ValueError("DifferentiableFit needs the module centres to align")
        x, y, z = (t.detach().contiguous() for t in (x, y, z))
        shift, rot = shift.detach().to(torch.float32).contiguous(), rot.detach().to(torch.float32).contiguous()
        xo, yo, zo = (torch.empty_like(x) for _ in range(3))
        L.align_hits(x.numel(), x.data_ptr(), y.data_ptr(), z.data_ptr(), self.module.data_ptr(),
                     self.centres.shape[0], self.centres.data_ptr(), shift.data_ptr(), rot.data_ptr(),
                     xo.data_ptr(), yo.data_ptr(), zo.data_ptr(), self._stream())
        return xo, yo, zo

    def _align_grad(self, x, y, z, rot, gxo, gyo, gzo, needs):
        x, y, z = (t.detach().contiguous() for t in (x, y, z))
        rot = rot.detach().to(torch.float32).contiguous()
        gxo, gyo, gzo = ((g if g is not None else torch.zeros_like(x)).contiguous() for g in (gxo, gyo, gzo))
        nm = self.centres.shape[0]
        want_hits = any(needs[:3])
        gx, gy, gz = ((torch.zeros_like(x) for _ in range(3)) if want_hits else (None, None, None))
        gs = torch.zeros(nm, 3, device=x.device) if needs[3] else None
        gr = torch.zeros(nm, 3, device=x.device) if needs[4] else None
        ptr = lambda t: None if t is None else t.data_ptr()
        L.align_hits_grad(x.numel(), x.data_ptr(), y.data_ptr(), z.data_ptr(), self.module.data_ptr(), nm,
                          self.centres.data_ptr(), rot.data_ptr(), gxo.data_ptr(), gyo.data_ptr(), gzo.data_ptr(),
                          ptr(gx), ptr(gy), ptr(gz), ptr(gs), ptr(gr), self._stream())
        return gx, gy, gz, gs, gr
