"""The learned warm start: training data from the solver itself, training with
the library's network kernels (dh_unet_backward / dh_unet_adam), and the
iterations it saves.  torch only holds device memory and slices batches; every
computation runs in libdehaze.so.

    net = WarmStartNet(base=32)
    data = make_dataset(256, 256, 256, seed0=5_000_000)
    net.train(data, steps=400, batch=8)
    print(evaluate(net, seeds=range(6_000_000, 6_000_008), H=256, W=256))
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _native as N
from . import api, scenes


def make_dataset(n: int, H: int, W: int, seed0: int, p=None, chunk: int = 64) -> dict:
    """n solver-generated training pairs: inputs (I, t, A, Phi), lambda and
    the target y* = lambda * u*, with u* the stable-preset solution to 1e-4
    (batched solve)."""
    p = p or api.params("stable")
    dev = torch.device("cuda")
    out = {k: [] for k in ("I", "t", "A", "Phi", "lam", "y")}
    for c0 in range(0, n, chunk):
        m = min(chunk, n - c0)
        Is = [torch.from_numpy(scenes.hazy_scene(seed0 + c0 + k, H, W)["I"]).to(dev) for k in range(m)]
        res = api.dehaze_batch(Is, p)
        for I, r in zip(Is, res):
            _, t, lam, Phi = api.transmission(I, r["A"], p)
            y = torch.empty_like(Phi)
            api._check(N.dh_warm_target(r["u"], lam, H, W, y, api._stream(None)), "dh_warm_target")
            for k, v in (("I", I), ("t", t), ("A", r["A"].clone()), ("Phi", Phi), ("lam", lam), ("y", y)):
                out[k].append(v)
    return {k: torch.stack(v) for k, v in out.items()}


class WarmStartNet:
    def __init__(self, base: int = 32, seed: int = 0, device="cuda"):
        self.base = base
        self.dev = torch.device(device)
        self.n = N.dh_unet_param_count(base)
        if self.n == 0:
            raise ValueError("base must be 16 or 32")
        self.params = torch.empty(self.n, device=self.dev)
        api._check(N.dh_unet_init(self.params, base, seed, api._stream(None)), "dh_unet_init")
        self._ws = {}

    def _workspace(self, n, H, W, train):
        key = (n, H, W, train)
        if key not in self._ws:
            nb = N.dh_unet_workspace_bytes(self.base, n, H, W, int(train))
            if nb == 0:
                raise ValueError("unsupported network shape (H, W multiples of 8)")
            self._ws[key] = torch.empty(nb, dtype=torch.uint8, device=self.dev)
        return self._ws[key]

    def train(self, data: dict, steps: int, batch: int = 8, lr: float = 1e-3, lr_end: float = 1e-4,
              log_every: int = 50, total_steps: int | None = None, seed: int = 12345) -> list:
        """Adam on mean((y - y*)^2); learning rate decays geometrically from
        lr to lr_end over total_steps (default: steps).  Batches cycle through
        the data in a fixed order.  The Adam moments and the step count persist
        across calls, so a run can go on with new data (chunked training)."""
        n, _, H, W = data["I"].shape
        total = total_steps or steps
        grads = torch.empty_like(self.params)
        if not hasattr(self, "_m"):
            self._m = torch.zeros_like(self.params)
            self._v = torch.zeros_like(self.params)
            self._step = 0
        loss = torch.empty(1, device=self.dev)
        ws = self._workspace(batch, H, W, True)
        log = []
        order = np.random.default_rng(seed).permutation(n)
        s = api._stream(None)
        for k in range(1, steps + 1):
            self._step += 1
            step = self._step
            idx = torch.from_numpy(order[[(k * batch + j) % n for j in range(batch)]]).to(self.dev)
            b = {key: data[key].index_select(0, idx).contiguous() for key in ("I", "t", "A", "Phi", "y")}
            api._check(N.dh_unet_backward(self.params, self.base, b["I"], b["t"], b["A"], b["Phi"], b["y"], batch, H,
                                          W, grads, loss, ws, ws.numel(), s), "dh_unet_backward")
            rate = lr * (lr_end / lr) ** (min(step - 1, total - 1) / max(1, total - 1))
            api._check(N.dh_unet_adam(self.params, grads, self._m, self._v, self.n, rate, 0.9, 0.999, 1e-8, step, s),
                       "dh_unet_adam")
            if k % log_every == 0 or k == 1 or k == steps:
                log.append((step, float(loss.item())))
        return log

    def predict(self, I, t, A, Phi):
        """y for a batch (N x 3 x H x W)."""
        n, _, H, W = I.shape
        y = torch.empty_like(Phi)
        ws = self._workspace(n, H, W, False)
        api._check(N.dh_unet_forward(self.params, self.base, I, t, A, Phi, n, H, W, y, ws, ws.numel(),
                                     api._stream(None)), "dh_unet_forward")
        return y

    def save(self, path: str):
        np.save(path, self.params.cpu().numpy())

    def load(self, path: str):
        self.params.copy_(torch.from_numpy(np.load(path)).to(self.dev))


class WarmDehazer:
    """dh_dehaze_warm for one image shape: front end, network warm start,
    fixed-point loop; workspaces kept resident."""

    def __init__(self, net: WarmStartNet, H: int, W: int, p=None):
        self.net, self.H, self.W = net, H, W
        self.p = p or api.params("stable")
        self.dz = api.Dehazer(H, W, self.p)
        self.nws = net._workspace(1, H, W, False)

    def __call__(self, I, report=True):
        rep = N.DhReport() if report else None
        rc = N.dh_dehaze_warm(self.net.params, self.net.base, I, self.H, self.W, self.p, self.dz.J, self.dz.u,
                              self.dz.t, self.dz.A, self.dz.ws, self.dz.ws.numel(), self.nws, self.nws.numel(),
                              api._stream(None), rep)
        api._check(rc, "dh_dehaze_warm")
        return rep


def analytic_u0(I, p=None):
    """u0 = Phi / lambda (the untrained network's guess), from the library."""
    p = p or api.params("stable")
    H, W = I.shape[1:]
    dc = api.dark_channel(I, p.patch)
    A, _, _ = api.atmospheric_light(I, dc, p.topk_permille)
    _, _, lam, Phi = api.transmission(I, A, p)
    u0 = torch.empty_like(Phi)
    api._check(N.dh_warm_start(Phi, lam, H, W, u0, api._stream(None)), "dh_warm_start")
    return u0


def evaluate(net: WarmStartNet | None, seeds, H: int, W: int, p=None, repeats: int = 3) -> dict:
    """Iterations and device time to the same residual from u0 = Phi (cold),
    u0 = Phi / lambda (analytic) and the network's u0, on held-out scenes."""
    p = p or api.params("stable")
    cold, ana, warm = api.Dehazer(H, W, p), api.Dehazer(H, W, p), None
    if net is not None:
        warm = WarmDehazer(net, H, W, p)
    rows = []
    for sd in seeds:
        I = torch.from_numpy(scenes.hazy_scene(sd, H, W)["I"]).cuda()
        r = {"seed": sd}
        for name, fn in (("cold", lambda: cold(I)), ("analytic", lambda: ana(I, analytic_u0(I, p))),
                         ("net", (lambda: warm(I)) if warm else None)):
            if fn is None:
                continue
            reps = [fn() for _ in range(repeats)]
            r[name] = {"n_iter": reps[-1].n_iter, "rho": max(reps[-1].rho), "ms": float(np.median([x.ms for x in reps]))}
        rows.append(r)
    summ = {}
    for name in ("cold", "analytic", "net"):
        if name in rows[0]:
            summ[name] = {"mean_iter": float(np.mean([r[name]["n_iter"] for r in rows])),
                          "mean_ms": float(np.mean([r[name]["ms"] for r in rows]))}
    return {"images": rows, "summary": summ}


def train_chunked(pairs: int, size: int, chunk: int, epochs: float = 1.0, batch: int = 8, base: int = 32,
                  lr: float = 1e-3, lr_end: float = 5e-5, seed0: int = 5_000_000, p=None) -> tuple:
    """Training on `pairs` solver-generated size x size scenes (seeds seed0 + i),
    generated and consumed `chunk` at a time so the set need not fit in
    memory; `epochs` passes over each chunk.  Returns (net, log, seconds)."""
    p = p or api.params("stable")
    net = WarmStartNet(base, seed=1)
    steps_per_chunk = max(1, int(round(epochs * chunk / batch)))
    nchunks = (pairs + chunk - 1) // chunk
    total = steps_per_chunk * nchunks
    log = []
    t0 = time.perf_counter()
    for c in range(nchunks):
        m = min(chunk, pairs - c * chunk)
        data = make_dataset(m, size, size, seed0=seed0 + c * chunk, p=p)
        log += net.train(data, steps_per_chunk, batch=batch, lr=lr, lr_end=lr_end,
                         log_every=steps_per_chunk, total_steps=total, seed=12345 + c)
        del data
    torch.cuda.synchronize()
    return net, log, time.perf_counter() - t0


def main():
    import argparse
    import json

    ap = argparse.ArgumentParser(description="chunked training of the warm-start network and its gain")
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--chunk", type=int, default=1000)
    ap.add_argument("--epochs", type=float, default=1.0)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--eval", type=int, default=4, help="held-out 1080p scenes (seeds 6e6 + i)")
    ap.add_argument("--save", default="", help="write the trained parameters (float32 .npy) and, beside "
                                               "them, a .json record of the run")
    a = ap.parse_args()
    net, log, secs = train_chunked(a.pairs, a.size, a.chunk, a.epochs, a.batch)
    ev = evaluate(net, range(6_000_000, 6_000_000 + a.eval), 1080, 1920)
    rec = {"pairs": a.pairs, "size": a.size, "chunk": a.chunk, "epochs": a.epochs, "batch": a.batch,
           "base": net.base, "train_s": secs, "loss_first": log[0][1], "loss_last": log[-1][1], "log": log,
           "eval_1080p": ev["summary"], "device": torch.cuda.get_device_name()}
    if a.save:
        net.save(a.save)
        with open(a.save[:-4] + ".json" if a.save.endswith(".npy") else a.save + ".json", "w") as f:
            json.dump(rec, f, indent=1)
    print(json.dumps({k: v for k, v in rec.items() if k != "log"}))


if __name__ == "__main__":
    main()
