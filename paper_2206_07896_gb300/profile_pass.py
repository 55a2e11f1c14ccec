"""One full-depth pass of the tuned stream kernel per tuning, for profilers.

    python -m paper_2206_07896_gb300.profile_pass N K:chunk:wpb:variant:stages [...]
    python -m paper_2206_07896_gb300.profile_pass vol N by:zchunks [...]
    python -m paper_2206_07896_gb300.profile_pass tileb N bx:by:depth [...]

Builds the N x N periodic FP32 workload (the seeded generator of the scale
runs), then launches, for each tuning given, ONE pass of depth K through
cpb_stencil_launch_tuned, so a profiler capturing `-k regex:stream -c <count>`
sees exactly one launch per tuning.  With `vol`: the N^3 volume workload and
ONE step of cpb_stencil3d_launch per geometry (block 32 x by, grid.z =
zchunks).  With `tileb`: the N x N periodic workload and ONE launch of depth
`depth` of cpb_stencil_tile_blocked per geometry.  Prints one line and exits 0.
"""
import sys


def main_vol(argv):
    import torch

    import workloads as W
    from . import lib

    n = int(argv[0]) if argv and ":" not in argv[0] else 256
    specs = [a for a in argv if ":" in a] or ["8:16"]
    L = lib(True)
    g = W.volume(n=n, steps=1)
    dev = torch.device("cuda")
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    out = torch.empty_like(u)
    for sp in specs:
        by, zc = (int(x) for x in sp.split(":"))
        L.cpb_stencil3d_launch(u, out, k, s, n, n, n, 1, float(g.dt), g.bc, ((n + 127) // 128, (n + by - 1) // by, zc),
                               (32, by, 1), L.cpb_stencil3d_shared_bytes(by))
    torch.cuda.synchronize()
    print("profile_pass vol", n, specs, "ok")
    return 0


def main_tileb(argv):
    import torch

    import workloads as W
    from . import lib

    n = int(argv[0]) if argv and ":" not in argv[0] else 4096
    specs = [a for a in argv if ":" in a] or ["64:16:8"]
    L = lib(True)
    g = W.plain_scale(seed=1, n=n, steps=1)
    dev = torch.device("cuda")
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    out, scr = torch.empty_like(u), torch.empty_like(u)
    for sp in specs:
        bx, by, d = (int(x) for x in sp.split(":"))
        L.cpb_stencil_tile_blocked(u, out, k, s, n, n, d, d, float(g.dt), g.bc,
                                   ((n + bx - 1) // bx, (n + by - 1) // by, 1), (bx, by, 1),
                                   L.cpb_tile_blocked_shared_bytes(bx, by, d), scratch=scr)
    torch.cuda.synchronize()
    print("profile_pass tileb", n, specs, "ok")
    return 0


def main(argv):
    if argv and argv[0] == "vol":
        return main_vol(argv[1:])
    if argv and argv[0] == "tileb":
        return main_tileb(argv[1:])
    import torch

    import workloads as W
    from . import lib

    n = int(argv[0]) if argv and ":" not in argv[0] else 4096
    specs = [a for a in argv if ":" in a] or ["4:256:1:1:2"]
    L = lib(True)
    g = W.plain_scale(seed=1, n=n, steps=16)
    dev = torch.device("cuda")
    u = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    s = torch.from_numpy(g.src).to(dev)
    out = torch.empty_like(u)
    for sp in specs:
        K, c, w, v, st = (int(x) for x in sp.split(":"))
        t = {"k": K, "chunk_rows": c, "warps_per_block": w, "variant": v, "stages": st}
        L.cpb_stencil_launch_tuned(u, out, k, s, n, n, K, float(g.dt), g.bc, 0, tuning=t)
    torch.cuda.synchronize()
    status = L.cpb_device_status()
    print("profile_pass", n, specs, "status", status)
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
