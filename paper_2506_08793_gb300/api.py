"""torch-tensor front end of the CUDA library (include/dehaze.h).

torch provides device memory and streams only; every step runs in the
library's kernels.  All functions raise on a library error and never fall back
to another implementation.
"""
from __future__ import annotations

import torch

from . import _native as N
from ._native import DhParams, DhReport


class DehazeError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {N.dh_strerror(status)} (status {status})")
        self.status = status


def _check(rc: int, where: str, ok=(N.DH_OK, N.DH_WDEGENERATE, N.DH_WNOCONV)) -> int:
    if rc not in ok:
        raise DehazeError(rc, where)
    return rc


def params(preset: str = "stable", **kw) -> DhParams:
    """Library parameters: preset 'paper' (the paper's constants) or 'stable'
    (eps = 1.0), then field overrides."""
    p = N.dh_params_default(N.DH_PRESET_PAPER if preset == "paper" else N.DH_PRESET_STABLE)
    return p.replace(**kw) if kw else p


def _img(I: torch.Tensor) -> tuple[int, int]:
    if I.dim() != 3 or I.shape[0] != 3 or I.dtype != torch.float32 or not I.is_cuda or not I.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor of shape (3, H, W)")
    return int(I.shape[1]), int(I.shape[2])


def _stream(stream):
    return torch.cuda.current_stream() if stream is None else stream


def workspace(H: int, W: int, p: DhParams, device) -> torch.Tensor:
    nb = N.dh_workspace_bytes(H, W, p)
    if nb == 0:
        raise ValueError("invalid shape or parameters")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def dark_channel(I: torch.Tensor, patch: int = 15, A: torch.Tensor | None = None, stream=None):
    H, W = _img(I)
    out = torch.empty((H, W), dtype=torch.float32, device=I.device)
    _check(N.dh_dark_channel(I, H, W, patch, A, out, _stream(stream)), "dh_dark_channel")
    return out


def atmospheric_light(I: torch.Tensor, dc: torch.Tensor, topk_permille: int = 1, stream=None):
    """Returns (A float32[3] on device, index int64[1] on device, report)."""
    H, W = _img(I)
    p = params("paper")
    ws = workspace(H, W, p, I.device)
    A = torch.empty(3, dtype=torch.float32, device=I.device)
    idx = torch.empty(1, dtype=torch.int64, device=I.device)
    rep = DhReport()
    _check(N.dh_atmospheric_light(I, dc, H, W, topk_permille, A, idx, ws, ws.numel(), _stream(stream), rep),
           "dh_atmospheric_light")
    return A, idx, rep


def transmission(I: torch.Tensor, A: torch.Tensor, p: DhParams | None = None, stream=None):
    """Returns (td, t, lambda, Phi)."""
    H, W = _img(I)
    p = p or params()
    td = torch.empty((H, W), dtype=torch.float32, device=I.device)
    t = torch.empty_like(td)
    lam = torch.empty_like(td)
    Phi = torch.empty_like(I)
    if p.dc_scales > 1 or p.gf_radius > 0:  # the refinements need workspace
        ws = workspace(H, W, p, I.device)
        _check(N.dh_transmission_ws(I, A, H, W, p, td, t, lam, Phi, ws, ws.numel(), _stream(stream)),
               "dh_transmission_ws")
    else:
        _check(N.dh_transmission(I, A, H, W, p, td, t, lam, Phi, _stream(stream)), "dh_transmission")
    return td, t, lam, Phi


def fixed_point(u: torch.Tensor, Phi: torch.Tensor, lam: torch.Tensor, p: DhParams | None = None,
                history: bool = False, stream=None):
    """Iterates u in place from u^0; returns (report, rho_hist or None)."""
    H, W = _img(u)
    p = p or params()
    ws = workspace(H, W, p, u.device)
    hist = torch.full((p.max_iter + 1, 3), float("nan"), device=u.device) if history else None
    rep = DhReport()
    _check(N.dh_fixed_point(u, Phi, lam, H, W, p, hist, ws, ws.numel(), _stream(stream), rep),
           "dh_fixed_point")
    return rep, hist


def semi_implicit(u: torch.Tensor, Phi: torch.Tensor, lam: torch.Tensor, p: DhParams | None = None,
                  step: float = 2.0, cg_iters: int = 32, history: bool = False, J: torch.Tensor | None = None,
                  u_lo: torch.Tensor | None = None, stream=None):
    """The semi-implicit (lagged-diffusivity) scheme in place on u from u^0
    (J, if given, receives clamp(u, 0, 1); u_lo, if given, is the trailing
    float32 part of the double-float iterate, in and out); returns (report,
    rho_hist or None).  Converges at the paper's eps = 1e-3."""
    H, W = _img(u)
    p = p or params("paper")
    ws = torch.empty(N.dh_semi_implicit_workspace_bytes(H, W), dtype=torch.uint8, device=u.device)
    hist = torch.full((p.max_iter + 1, 3), float("nan"), device=u.device) if history else None
    rep = DhReport()
    _check(N.dh_semi_implicit(u, u_lo, Phi, lam, H, W, p, step, cg_iters, hist, J, ws, ws.numel(),
                              _stream(stream), rep), "dh_semi_implicit")
    return rep, hist


def dehaze_semi_implicit(I: torch.Tensor, p: DhParams | None = None, step: float = 2.0, cg_iters: int = 32):
    """The whole method with the semi-implicit solver: dark channel, A, t,
    lambda, Phi, then the scheme from u^0 = Phi.  Returns a dict like dehaze()."""
    p = p or params("paper")
    dc = dark_channel(I, p.patch)
    A, idx, _ = atmospheric_light(I, dc, p.topk_permille)
    _, t, lam, Phi = transmission(I, A, p)
    u = Phi.clone()
    J = torch.empty_like(u)
    rep, _ = semi_implicit(u, Phi, lam, p, step, cg_iters, J=J)
    return {"J": J, "u": u, "t": t, "A": A, "report": rep}


class Dehazer:
    """The whole method for images of one shape, with the workspace and the
    outputs kept resident so that repeated calls reuse the cached loop graph."""

    def __init__(self, H: int, W: int, p: DhParams | None = None, device="cuda"):
        self.H, self.W = H, W
        self.p = p or params()
        self.device = torch.device(device)
        self.ws = workspace(H, W, self.p, self.device)
        self.J = torch.empty((3, H, W), dtype=torch.float32, device=self.device)
        self.u = torch.empty_like(self.J)
        self.t = torch.empty((H, W), dtype=torch.float32, device=self.device)
        self.A = torch.empty(3, dtype=torch.float32, device=self.device)

    def __call__(self, I: torch.Tensor, u0: torch.Tensor | None = None, report: bool = True, stream=None):
        H, W = _img(I)
        if (H, W) != (self.H, self.W):
            raise ValueError("image shape differs from the Dehazer's")
        rep = DhReport() if report else None
        rc = N.dh_dehaze(I, H, W, self.p, u0, self.J, self.u, self.t, self.A, self.ws, self.ws.numel(),
                         _stream(stream), rep)
        _check(rc, "dh_dehaze")
        return rep


def dehaze(I: torch.Tensor, p: DhParams | None = None, u0: torch.Tensor | None = None):
    """One image: returns dict(J, u, t, A, report)."""
    H, W = _img(I)
    d = Dehazer(H, W, p, I.device)
    rep = d(I, u0)
    return dict(J=d.J, u=d.u, t=d.t, A=d.A, report=rep)


class BatchDehazer:
    """The whole method on a fixed list of image shapes, solved together: one
    persistent sweep launch per iteration over every image still iterating.
    Outputs and workspace stay resident between calls."""

    def __init__(self, shapes, p: DhParams | None = None, device="cuda", net=None):
        """net: a warm-start network (an object with .params, a float32 CUDA
        tensor, and .base, e.g. warmstart.WarmStartNet); with it every image
        starts from the network's u0 (dh_dehaze_batch_warm)."""
        import ctypes

        self.net = net
        self.shapes = [tuple(map(int, s)) for s in shapes]
        self.p = p or params()
        self.device = torch.device(device)
        self.out = []
        for H, W in self.shapes:
            self.out.append(dict(J=torch.empty((3, H, W), dtype=torch.float32, device=self.device),
                                 u=torch.empty((3, H, W), dtype=torch.float32, device=self.device),
                                 t=torch.empty((H, W), dtype=torch.float32, device=self.device),
                                 A=torch.empty(3, dtype=torch.float32, device=self.device)))
        self._reports = (DhReport * len(self.shapes))()
        probe = [N.dh_image(None, H, W, None, o["J"], o["u"], o["t"], o["A"])
                 for (H, W), o in zip(self.shapes, self.out)]
        nb = N.dh_batch_workspace_bytes(len(probe), probe, self.p)
        if nb == 0:
            raise ValueError("invalid batch")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.nws = None
        if net is not None:
            nn = N.dh_batch_net_workspace_bytes(net.base, len(probe), probe)
            if nn == 0:
                raise ValueError("the network takes image sides that are multiples of 8")
            self.nws = torch.empty(nn, dtype=torch.uint8, device=self.device)
        self._ctypes = ctypes

    def __call__(self, images, u0s=None, report: bool = True, stream=None):
        if len(images) != len(self.shapes):
            raise ValueError("wrong number of images")
        imgs = []
        for k, (I, (H, W), o) in enumerate(zip(images, self.shapes, self.out)):
            if _img(I) != (H, W):
                raise ValueError(f"image {k} has the wrong shape")
            u0 = None if u0s is None else u0s[k]
            imgs.append(N.dh_image(I, H, W, u0, o["J"], o["u"], o["t"], o["A"]))
        reps = self._reports if report else None
        if self.net is not None:
            if u0s is not None:
                raise ValueError("a warm-started batch takes its u0 from the network")
            rc = N.dh_dehaze_batch_warm(self.net.params, self.net.base, len(imgs), imgs, self.p, self.ws,
                                        self.ws.numel(), self.nws, self.nws.numel(), _stream(stream), reps)
            _check(rc, "dh_dehaze_batch_warm")
        else:
            rc = N.dh_dehaze_batch(len(imgs), imgs, self.p, self.ws, self.ws.numel(), _stream(stream), reps)
            _check(rc, "dh_dehaze_batch")
        return [DhReport.from_buffer_copy(r) for r in self._reports] if report else None


def dehaze_batch(images, p: DhParams | None = None):
    """Several images of any sizes in one batched solve; returns one dict per
    image (J, u, t, A, report)."""
    b = BatchDehazer([tuple(I.shape[1:]) for I in images], p, images[0].device)
    reps = b(images)
    return [dict(o, report=r) for o, r in zip(b.out, reps)]


def tune(I: torch.Tensor, p: DhParams | None = None, iters: int = 40) -> dict:
    """Times every sweep variant on this image's own Phi and lambda and records
    the fastest for its shape (used by later calls on this device).  Returns
    {"best": id, "us_per_iter": {id: us}}."""
    H, W = _img(I)
    p = p or params()
    dc = dark_channel(I, p.patch)
    A, _, _ = atmospheric_light(I, dc, p.topk_permille)
    _, _, lam, Phi = transmission(I, A, p)
    ws = workspace(H, W, p, I.device)
    u = torch.empty_like(Phi)
    res = N.DhTuneResult()
    _check(N.dh_tune(Phi, lam, u, H, W, p, iters, ws, ws.numel(), _stream(None), res), "dh_tune")
    return {"best": res.best, "us_per_iter": {res.variant[k]: res.us_per_iter[k] for k in range(res.count)}}


def save_tuning(path: str, shapes) -> None:
    """Writes the tuned variants of these (H, W) shapes (float32 storage) as JSON."""
    import json

    table = {f"{H}x{W}": N.dh_tune_get(H, W, N.DH_STORE_F32) for H, W in shapes}
    with open(path, "w") as f:
        json.dump({"device": torch.cuda.get_device_name(), "variants": table}, f, indent=1)


def load_tuning(path: str) -> int:
    """Loads a JSON tuning table written by save_tuning into the library;
    returns the number of entries applied (0 when it was made on another GPU)."""
    import json

    with open(path) as f:
        t = json.load(f)
    if t.get("device") != torch.cuda.get_device_name():
        return 0
    n = 0
    for key, v in t["variants"].items():
        H, W = map(int, key.split("x"))
        if v and N.dh_tune_set(H, W, N.DH_STORE_F32, int(v)) == N.DH_OK:
            n += 1
    return n
