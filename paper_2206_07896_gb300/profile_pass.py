"""One full-depth pass of the tuned stream kernel per tuning, for profilers.

    python -m paper_2206_07896_gb300.profile_pass N K:chunk:wpb:variant:stages [...]
    python -m paper_2206_07896_gb300.profile_pass vol N by:zchunks [...]
    python -m paper_2206_07896_gb300.profile_pass tileb N bx:by:depth [...]
    python -m paper_2206_07896_gb300.profile_pass adjoint
    python -m paper_2206_07896_gb300.profile_pass batch NGRIDS

Builds the N x N periodic FP32 workload (the seeded generator of the scale
runs), then launches, for each tuning given, ONE pass of depth K through
cpb_stencil_launch_tuned, so a profiler capturing `-k regex:stream -c <count>`
sees exactly one launch per tuning.  With `vol`: the N^3 volume workload and
ONE step of cpb_stencil3d_launch per geometry (block 32 x by, grid.z =
zchunks).  With `tileb`: the N x N periodic workload and ONE launch of depth
`depth` of cpb_stencil_tile_blocked per geometry.  With `adjoint`: ONE
gradient of the 2048^2 differentiation workload (checkpointed forward, then
the backward sweep with segment recompute), as the bench times it.  With
`batch`: ONE batched persistent launch over the NGRIDS cheapest grids (by
cell-updates) of the 4096-grid set, default plan; a subset of cheap grids
keeps every grid far below the per-SM share of the work, so that no single
grid sets the length of the launch.  Prints one line and exits 0 (1 on a non-zero
device status).
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


def main_adjoint(argv):
    import torch

    import workloads as W
    from . import lib

    L = lib(True)
    g = W.differentiation()
    dev = torch.device("cuda")
    nx, ny, T, ck = g.nx, g.ny, g.steps, g.extras["ckpt"]
    u0 = torch.from_numpy(g.u).to(dev)
    k = torch.from_numpy(g.kappa).to(dev)
    tgt = torch.from_numpy(g.extras["target"]).to(dev)
    wsb = L.cpb_adjoint_workspace_bytes(nx, ny, T, ck)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    uT, gu, gk = torch.empty_like(u0), torch.empty_like(u0), torch.empty_like(u0)
    L.cpb_adjoint_forward(u0, k, None, nx, ny, T, float(g.dt), g.bc, ck, uT, ws, wsb)
    lam = uT - tgt
    L.cpb_adjoint_backward(k, None, lam, nx, ny, T, float(g.dt), g.bc, ck, gu, gk, ws, wsb)
    torch.cuda.synchronize()
    status = L.cpb_device_status()
    print("profile_pass adjoint", g.name, "status", status)
    return 0 if status == 0 else 1


def main_batch(argv):
    import ctypes as C

    import numpy as np
    import torch

    import workloads as W
    from . import batch_descriptors, lib, to_device_bytes, CPB_F32

    n = int(argv[0]) if argv else 512
    L = lib(True)
    bt = W.batching(ngrids=4096)
    sel = np.sort(np.argsort(bt.nx.astype(np.int64) * bt.ny * bt.steps, kind="stable")[:n])
    nx, ny, steps, dt = bt.nx[sel], bt.ny[sel], bt.steps[sel], bt.dt[sel]
    cells = nx.astype(np.int64) * ny.astype(np.int64)
    off = np.zeros(n, np.int64)
    off[1:] = np.cumsum((cells + 3) // 4 * 4)[:-1]  # 16-byte aligned grid starts
    total = int(off[-1] + cells[-1])
    dev = torch.device("cuda")
    u = torch.zeros(total, dtype=torch.float32, device=dev)
    k = torch.ones(total, dtype=torch.float32, device=dev)
    s = torch.zeros(total, dtype=torch.float32, device=dev)
    for q, g in enumerate(sel):
        o, c, b = int(off[q]), int(cells[q]), int(bt.offset[g])
        u[o:o + c] = torch.from_numpy(bt.u[b:b + c])
        k[o:o + c] = torch.from_numpy(bt.kappa[b:b + c])
        s[o:o + c] = torch.from_numpy(bt.src[b:b + c])
    uo = torch.empty_like(u)
    descs = batch_descriptors(u, uo, k, s, off, nx, ny, steps, dt)
    plan = L.cpb_batch_plan_default()
    order, n_large = L.cpb_batch_order(descs, plan)
    d_descs = to_device_bytes(descs, dev)
    d_order = to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    L.cpb_stencil_batched(d_descs, d_order, n, n_large, CPB_F32, W.DIRICHLET, plan, work)
    torch.cuda.synchronize()
    status = L.cpb_batch_status(work)
    print("profile_pass batch", n, "grids", int((cells * steps.astype(np.int64)).sum()), "updates status",
          status)
    return 0 if status == 0 else 1


def main(argv):
    if argv and argv[0] == "adjoint":
        return main_adjoint(argv[1:])
    if argv and argv[0] == "batch":
        return main_batch(argv[1:])
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
