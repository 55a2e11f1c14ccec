"""GPU parity of the batched persistent launch (many uneven grids, one launch)."""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
cpb = pytest.importorskip("paper_2206_07896_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def small_batch(seed, bc):
    rng = np.random.default_rng(seed)
    shapes = [(1, 1), (1, 200), (200, 1), (3, 5), (128, 128), (300, 70), (64, 64), (257, 33)]
    shapes += [(int(a), int(b)) for a, b in rng.integers(1, 260, (40, 2))]
    steps = [int(x) for x in rng.integers(0, 26, len(shapes))]
    steps[0], steps[1] = 0, 1
    grids = [W.random_grid(seed * 1000 + i, nx, ny, st, bc) for i, ((nx, ny), st) in
             enumerate(zip(shapes, steps))]
    return grids


def pack(grids, dev):
    sizes = [g.nx * g.ny for g in grids]
    off = np.zeros(len(grids), np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    # pad each grid start to 16 bytes so most grids take the 128-bit path
    off = np.array([((o + 3) // 4) * 4 + 4 * i for i, o in enumerate(off)], np.int64)
    total = int(off[-1] + sizes[-1] + 8)
    u = torch.zeros(total, dtype=torch.float32, device=dev)
    k = torch.ones(total, dtype=torch.float32, device=dev)
    s = torch.zeros(total, dtype=torch.float32, device=dev)
    for g, o in zip(grids, off):
        n = g.nx * g.ny
        u[o:o + n] = torch.from_numpy(g.u.reshape(-1)).to(dev)
        k[o:o + n] = torch.from_numpy(g.kappa.reshape(-1)).to(dev)
        s[o:o + n] = torch.from_numpy(g.src.reshape(-1)).to(dev)
    return u, k, s, off


def run_batch(L, grids, dev, bc, plan, u, k, s, off):
    uo = torch.full_like(u, -1.0)
    uin = u.clone()
    descs = cpb.batch_descriptors(uin, uo, k, s, off, [g.nx for g in grids], [g.ny for g in grids],
                                  [g.steps for g in grids], [g.dt for g in grids])
    order, n_large = L.cpb_batch_order(descs, plan)
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    L.cpb_stencil_batched(d_descs, d_order, len(grids), n_large, cpb.CPB_F32, bc, plan, work)
    assert L.cpb_batch_status(work) == 0
    return uo, n_large


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.PERIODIC])
@pytest.mark.parametrize("plan", [{"grain": 1, "blocks": 0, "threads": 384, "team_cells": 4096},
                                  {"grain": 3, "blocks": 3, "threads": 256, "team_cells": 20000},
                                  {"grain": 2, "blocks": 0, "threads": 128, "team_cells": 1},
                                  {"grain": 1, "blocks": 0, "threads": 256, "team_cells": 4096, "depth": 8},
                                  {"grain": 2, "blocks": 5, "threads": 128, "team_cells": 20000,
                                   "depth": 8},
                                  {"grain": 1, "blocks": 0, "threads": 384, "team_cells": 20000, "team_warps": 4},
                                  {"grain": 2, "blocks": 4, "threads": 384, "team_cells": 4096, "team_warps": 3},
                                  {"grain": 1, "blocks": 0, "threads": 256, "team_cells": 1 << 30, "team_warps": 2,
                                   "depth": 8},
                                  {"grain": 1, "blocks": 3, "threads": 384, "team_cells": 1 << 30, "team_warps": 12}])
def test_batched_bit_exact(dev, bc, plan):
    L = cpb.lib(fma=False)
    grids = small_batch(7 + bc, bc)
    u, k, s, off = pack(grids, dev)
    uo, n_large = run_batch(L, grids, dev, bc, plan, u, k, s, off)
    assert 0 < n_large < len(grids) or plan["team_cells"] in (1, 1 << 30)
    out = uo.cpu().numpy()
    for g, o in zip(grids, off):
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
        got = out[o:o + g.nx * g.ny].reshape(g.ny, g.nx)
        np.testing.assert_array_equal(got, ref, err_msg=f"{g.nx}x{g.ny} steps={g.steps}")


def test_batch_order_is_lpt_and_validates(dev):
    L = cpb.lib(fma=False)
    grids = small_batch(3, W.DIRICHLET)
    u, k, s, off = pack(grids, dev)
    descs = cpb.batch_descriptors(u, torch.empty_like(u), k, s, off, [g.nx for g in grids],
                                  [g.ny for g in grids], [g.steps for g in grids],
                                  [g.dt for g in grids])
    plan = {"grain": 1, "team_cells": 4096}
    order, n_large = L.cpb_batch_order(descs, plan)
    assert sorted(order) == list(range(len(grids)))
    cost = [g.nx * g.ny * g.steps for g in grids]
    big = [i for i in order[:n_large]]
    assert all(grids[i].nx * grids[i].ny >= 4096 for i in big)
    assert all(cost[a] >= cost[b] for a, b in zip(big, big[1:]))
    small = order[n_large:]
    assert all(cost[a] >= cost[b] for a, b in zip(small, small[1:]))
    descs[5].nx = 0
    with pytest.raises(cpb.CpbError) as e:
        L.cpb_batch_order(descs, plan)
    assert e.value.status == cpb.CPB_ERR_INVALID_VALUE


def test_batched_invalid_device_descriptor_is_reported(dev):
    L = cpb.lib(fma=False)
    grids = small_batch(5, W.PERIODIC)[:10]
    u, k, s, off = pack(grids, dev)
    uo = torch.full_like(u, -1.0)
    uin = u.clone()                   # keep a reference: the descriptors hold raw pointers
    descs = cpb.batch_descriptors(uin, uo, k, s, off, [g.nx for g in grids],
                                  [g.ny for g in grids], [g.steps for g in grids],
                                  [g.dt for g in grids])
    order, n_large = L.cpb_batch_order(descs, None)
    descs[order[-1]].ny = -3          # corrupt only the device copy
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    L.cpb_stencil_batched(d_descs, d_order, len(grids), n_large, cpb.CPB_F32, W.PERIODIC, None, work)
    assert L.cpb_batch_status(work) == cpb.CPB_ERR_INVALID_VALUE
    out = uo.cpu().numpy()
    for i, (g, o) in enumerate(zip(grids, off)):
        if i == order[-1]:
            continue
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, W.PERIODIC, "f32")
        np.testing.assert_array_equal(out[o:o + g.nx * g.ny].reshape(g.ny, g.nx), ref)


def test_batched_graph_capture(dev):
    L = cpb.lib(fma=False)
    grids = small_batch(11, W.DIRICHLET)[:20]
    u, k, s, off = pack(grids, dev)
    uo = torch.zeros_like(u)
    uin = u.clone()
    descs = cpb.batch_descriptors(uin, uo, k, s, off, [g.nx for g in grids], [g.ny for g in grids],
                                  [g.steps for g in grids], [g.dt for g in grids])
    order, n_large = L.cpb_batch_order(descs, None)
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    s_ = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s_):
        L.cpb_stencil_batched(d_descs, d_order, len(grids), n_large, cpb.CPB_F32, W.DIRICHLET, None,
                              work, stream=s_)
    for _ in range(2):
        uin.copy_(u)       # the batch clobbers u_in; restore it before each replay
        uo.zero_()
        graph.replay()
        torch.cuda.synchronize()
        out = uo.cpu().numpy()
        for g, o in zip(grids, off):
            ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, W.DIRICHLET, "f32")
            np.testing.assert_array_equal(out[o:o + g.nx * g.ny].reshape(g.ny, g.nx), ref)


@pytest.mark.parametrize("depth", [4, 8])   # single rows / rows in pairs
def test_batched_ring_timeout_falls_back_and_is_reported(dev, depth):
    # One row's copies never complete (test hook) with a short wait limit:
    # the warps that meet it report CPB_ERR_TIMEOUT, redo the item with
    # ordinary loads, and every grid's result is still exact.
    L = cpb.lib(fma=False)
    grids = [W.random_grid(40 + i, nx, ny, st, W.PERIODIC)
             for i, (nx, ny, st) in enumerate([(256, 40, 9), (128, 30, 6), (512, 20, 5), (96, 50, 7)])]
    u, k, s, off = pack(grids, dev)
    plan = {"grain": 1, "blocks": 2, "threads": 128, "team_cells": 6000, "depth": depth}
    uo = torch.full_like(u, -1.0)
    uin = u.clone()
    descs = cpb.batch_descriptors(uin, uo, k, s, off, [g.nx for g in grids],
                                  [g.ny for g in grids], [g.steps for g in grids],
                                  [g.dt for g in grids])
    order, n_large = L.cpb_batch_order(descs, plan)
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    try:
        L.cpb_debug_set(2000, 7)
        L.cpb_stencil_batched(d_descs, d_order, len(grids), n_large, cpb.CPB_F32, W.PERIODIC, plan,
                              work)
        assert L.cpb_batch_status(work) == cpb.CPB_ERR_TIMEOUT
    finally:
        L.cpb_debug_set(0, -1)
    out = uo.cpu().numpy()
    for g, o in zip(grids, off):
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, W.PERIODIC, "f32")
        np.testing.assert_array_equal(out[o:o + g.nx * g.ny].reshape(g.ny, g.nx), ref)
    # the next launch, without the hook, is clean
    uin.copy_(u)
    L.cpb_stencil_batched(d_descs, d_order, len(grids), n_large, cpb.CPB_F32, W.PERIODIC, plan, work)
    assert L.cpb_batch_status(work) == 0


def test_batch_autotune_picks_a_measured_plan_that_stays_exact(dev):
    # Grain-size selection (the GPU counterpart of average vs aggressive
    # coarse-grained fetching): every candidate is timed, the chosen plan is
    # one of them, and a run with it is still bit-exact.
    L = cpb.lib(fma=False)
    bc = W.DIRICHLET
    grids = small_batch(17, bc)
    u, k, s, off = pack(grids, dev)
    plan0 = {"grain": 1, "blocks": 0, "threads": 384, "team_cells": 4096}
    # tune on copies: the tuning runs overwrite u_in and u_out
    tu, to = u.clone(), torch.empty_like(u)
    descs = cpb.batch_descriptors(tu, to, k, s, off, [g.nx for g in grids], [g.ny for g in grids],
                                  [g.steps for g in grids], [g.dt for g in grids])
    order, n_large = L.cpb_batch_order(descs, plan0)
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    best, table = L.cpb_batch_autotune(d_descs, d_order, len(grids), n_large, cpb.CPB_F32, bc, work,
                                       plan0)
    assert len(table) == cpb.BATCH_TUNE_CANDIDATES
    for (d, g, t), v in table.items():
        if d == 8 and t > 256:
            assert v is None                 # not a valid plan at depth 8
        else:
            assert v is not None and v > 0
    assert table[(best["depth"], best["grain"], best["threads"])] is not None
    assert best["team_cells"] == plan0["team_cells"] and best["blocks"] == 0
    uo, _ = run_batch(L, grids, dev, bc, best, u, k, s, off)
    out = uo.cpu().numpy()
    for g, o in zip(grids, off):
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
        np.testing.assert_array_equal(out[o:o + g.nx * g.ny].reshape(g.ny, g.nx), ref)


@pytest.mark.slow
def test_full_batching_workload_sampled_grids_bit_exact(dev):
    # The batching workload as the benchmark runs it: all 4096 grids packed
    # back to back (each start on a 16-byte boundary), the grain / CTA-size
    # plan chosen by the batched autotuner, one persistent launch.  Sampled
    # grids (the most expensive, the cheapest, the widest, the narrowest and a
    # seeded spread) equal the FP32 oracle bit for bit (--fmad=false build).
    L = cpb.lib(fma=False)
    bt = W.batching()
    cells = bt.nx.astype(np.int64) * bt.ny.astype(np.int64)
    off = np.zeros(bt.ngrids, np.int64)
    off[1:] = np.cumsum((cells + 3) // 4 * 4)[:-1]
    total = int(off[-1] + cells[-1])
    u = torch.zeros(total, dtype=torch.float32, device=dev)
    k = torch.ones(total, dtype=torch.float32, device=dev)
    s = torch.zeros(total, dtype=torch.float32, device=dev)
    for g in range(bt.ngrids):
        o, c, b = int(off[g]), int(cells[g]), int(bt.offset[g])
        u[o:o + c] = torch.from_numpy(bt.u[b:b + c])
        k[o:o + c] = torch.from_numpy(bt.kappa[b:b + c])
        s[o:o + c] = torch.from_numpy(bt.src[b:b + c])
    tu, to = u.clone(), torch.empty_like(u)
    descs = cpb.batch_descriptors(tu, to, k, s, off, bt.nx, bt.ny, bt.steps, bt.dt)
    plan = L.cpb_batch_plan_default()
    order, n_large = L.cpb_batch_order(descs, plan)
    d_descs = cpb.to_device_bytes(descs, dev)
    d_order = cpb.to_device_bytes((C.c_int * len(order))(*order), dev)
    work = torch.zeros(4, dtype=torch.int32, device=dev)
    plan, _ = L.cpb_batch_autotune(d_descs, d_order, bt.ngrids, n_large, cpb.CPB_F32, W.DIRICHLET, work, plan)
    del tu, to
    uo = torch.full_like(u, -1.0)
    uin = u.clone()
    descs = cpb.batch_descriptors(uin, uo, k, s, off, bt.nx, bt.ny, bt.steps, bt.dt)
    d_descs = cpb.to_device_bytes(descs, dev)
    L.cpb_stencil_batched(d_descs, d_order, bt.ngrids, n_large, cpb.CPB_F32, W.DIRICHLET, plan, work)
    assert L.cpb_batch_status(work) == 0
    out = uo.cpu().numpy()
    cost = cells * bt.steps.astype(np.int64)
    rng = np.random.default_rng(7)
    sample = set(np.argsort(cost)[-4:]) | set(np.argsort(cost)[:4]) | {int(np.argmax(bt.nx)), int(np.argmin(bt.nx))}
    sample |= set(int(x) for x in rng.choice(bt.ngrids, 18, replace=False))
    for gi in sorted(sample):
        g = bt.grid(int(gi))
        ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, W.DIRICHLET, "f32", pool=oracle.host_cores())
        o = int(off[gi])
        np.testing.assert_array_equal(out[o:o + g.nx * g.ny].reshape(g.ny, g.nx), ref, err_msg=f"grid {gi}")
