"""A fixed, small workload for profilers: the whole method on one synthetic
scene with a fixed number of fixed-point iterations (tol = 0), so the sweep
kernel runs exactly iters + 1 times.

    python -m paper_2506_08793_gb300.profile_case --H 1080 --W 1920 --iters 8
"""
import argparse

import torch

from . import api, scenes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--H", type=int, default=1080)
    ap.add_argument("--W", type=int, default=1920)
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--preset", default="stable")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--storage", type=int, default=0, help="0 f32, 1 bf16, 2 f16, 3 bf16->f32, 4 f16->f32")
    ap.add_argument("--tol", type=float, default=0.0)
    ap.add_argument("--variant", type=int, default=0, help="sweep variant (0: library default)")
    ap.add_argument("--net", type=int, default=0, help="instead: N images through the warm-start network forward")
    ap.add_argument("--conv", default="", help="instead: one 3x3 convolution 'C,Cout' on 1 x H x W, --repeat times")
    ap.add_argument("--wgrad", default="", help="instead: the weight gradient of one 3x3 convolution 'C,Cout' "
                                                "on 1 x H x W, --repeat times")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead: N images of the mixed photo sizes (seed 3000) in one batched solve")
    ap.add_argument("--semi", type=int, default=0,
                    help="instead: the semi-implicit solver with this many CG iterations per outer step "
                         "(paper preset, --iters outer steps)")
    ap.add_argument("--host-loop", action="store_true",
                    help="queue the sweeps from the host instead of the graph loop (profilers cannot "
                         "see kernels inside a graph with conditional nodes)")
    a = ap.parse_args()
    if a.batch:
        sizes = scenes.batch_sizes(3000, a.batch)
        imgs = [torch.from_numpy(scenes.hazy_scene(3000 + k, H, W)["I"]).cuda() for k, (H, W) in enumerate(sizes)]
        b = api.BatchDehazer(sizes, api.params(a.preset, tol=a.tol, max_iter=a.iters,
                                               use_graph=0 if a.host_loop else 1))
        for _ in range(a.repeat):
            reps = b(imgs)
        torch.cuda.synchronize()
        print(f"batch of {a.batch}: {[r.n_iter for r in reps]} iterations, {reps[0].ms:.3f} ms")
        return
    if a.semi:
        I = torch.from_numpy(scenes.hazy_scene(a.seed, a.H, a.W)["I"]).cuda()
        p = api.params("paper", tol=a.tol, max_iter=a.iters)
        dc = api.dark_channel(I, p.patch)
        A, _, _ = api.atmospheric_light(I, dc, p.topk_permille)
        _, _, lam, Phi = api.transmission(I, A, p)
        for _ in range(a.repeat):
            u = Phi.clone()
            rep, _ = api.semi_implicit(u, Phi, lam, p, 2.0, a.semi)
        torch.cuda.synchronize()
        print(f"semi-implicit {a.H}x{a.W}: {rep.n_iter} outer steps, {rep.ms:.3f} ms, status {rep.status}")
        return
    if a.conv:
        from . import _native as N

        C, Cout = (int(v) for v in a.conv.split(","))
        g = torch.Generator().manual_seed(a.seed)
        x = (torch.rand(a.H * a.W * C, generator=g) - 0.5).to(torch.bfloat16).cuda()
        w = ((torch.rand(Cout * 9 * C, generator=g) - 0.5) * 0.1).to(torch.bfloat16).cuda()
        b = torch.zeros(Cout, device="cuda")
        y = torch.empty(a.H * a.W * Cout, dtype=torch.bfloat16, device="cuda")
        for _ in range(a.repeat):
            rc = N.dh_conv3x3_forward(x, C, C, 1, a.H, a.W, w, b, Cout, 1, y, Cout)
            if rc:
                raise SystemExit(f"dh_conv3x3_forward: {rc}")
        torch.cuda.synchronize()
        print(f"conv {C}->{Cout} on {a.H}x{a.W} x{a.repeat}: done")
        return
    if a.wgrad:
        from . import _native as N

        C, Cout = (int(v) for v in a.wgrad.split(","))
        g = torch.Generator().manual_seed(a.seed)
        x = (torch.rand(a.H * a.W * C, generator=g) - 0.5).to(torch.bfloat16).cuda()
        dy = (torch.rand(a.H * a.W * Cout, generator=g) - 0.5).to(torch.bfloat16).cuda()
        dw = torch.empty(Cout * 9 * C, device="cuda")
        db = torch.empty(Cout, device="cuda")
        scratch = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        for _ in range(a.repeat):
            rc = N.dh_conv3x3_backward_weights(x, C, C, dy, Cout, Cout, 1, a.H, a.W, dw, db, scratch, scratch.numel())
            if rc:
                raise SystemExit(f"dh_conv3x3_backward_weights: {rc}")
        torch.cuda.synchronize()
        print(f"weight gradient {C}->{Cout} on {a.H}x{a.W} x{a.repeat}: done")
        return
    if a.net:
        from . import warmstart as WS

        net = WS.WarmStartNet(32, seed=1)
        I = torch.stack([torch.from_numpy(scenes.hazy_scene(a.seed + k, a.H, a.W)["I"]) for k in range(a.net)]).cuda()
        t = torch.rand((a.net, a.H, a.W), device="cuda")
        A = torch.rand((a.net, 3), device="cuda")
        for _ in range(a.repeat):
            y = net.predict(I, t, A, I)
        torch.cuda.synchronize()
        print(f"network forward on {a.net} x {a.H}x{a.W}: done")
        return
    I = torch.from_numpy(scenes.hazy_scene(a.seed, a.H, a.W)["I"]).cuda()
    d = api.Dehazer(a.H, a.W, api.params(a.preset, tol=a.tol, max_iter=a.iters, storage=a.storage,
                                                   use_graph=0 if a.host_loop else 1, sweep_variant=a.variant))
    for _ in range(a.repeat):
        rep = d(I)
    torch.cuda.synchronize()
    print(f"{a.H}x{a.W}: {rep.n_iter} iterations, {rep.ms:.3f} ms, loop {rep.ms_loop:.3f} ms, "
          f"{rep.launches} launches, status {rep.status}, rho {max(rep.rho):.3e}")


if __name__ == "__main__":
    main()
