"""Pins for the oracle's stencil arithmetic, each against something other than itself.

The update is the flux-form 5-point step (a stated reading; the paper has no
stencil): u' = c + (hdt * ((fW + fE) + (fS + fN)) + dt * s), f = (kc + kn)(un - c),
hdt = dt / 2; Dirichlet ghosts have u = 0 and kappa = kc; periodic wraps.

Pins used here:
* exact rational arithmetic through an operator assembled face by face,
* closed-form Fourier / sine-mode decay factors,
* exact conservation, constant-source growth, the maximum principle,
* bit-exact mirror and transpose symmetry,
* the tiled kernel executed with loop fission equals the direct loop bit for bit,
* bf16 rounding against torch's conversion,
* FP64 heat sum against an exactly rounded sum (math.fsum),
* the adjoint against central finite differences.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

D, P = W.DIRICHLET, W.PERIODIC


# ---------------------------------------------------------------------------
# brute force in exact arithmetic
# ---------------------------------------------------------------------------
def exact_operator(kappa, bc, hdt):
    """64x64 (or nx*ny square) operator A with u' = A u + dt s, exact Fractions.

    Assembled per face, independently of the per-cell formula: a face between
    cells p and q with conductivity hdt*(k_p + k_q) moves heat from the hotter
    to the colder one; a Dirichlet boundary face of cell p has conductivity
    hdt*(2 k_p) towards a ghost held at zero.
    """
    ny, nx = kappa.shape
    n = nx * ny
    A = [[Fraction(0)] * n for _ in range(n)]
    for p in range(n):
        A[p][p] = Fraction(1)
    K = [[Fraction(float(kappa[j, i])) for i in range(nx)] for j in range(ny)]
    faces = []
    for j in range(ny):
        for i in range(nx):
            if i + 1 < nx:
                faces.append(((i, j), (i + 1, j)))
            elif bc == P:
                faces.append(((i, j), (0, j)))
            if j + 1 < ny:
                faces.append(((i, j), (i, j + 1)))
            elif bc == P:
                faces.append(((i, j), (i, 0)))
    for (i, j), (a, b) in faces:
        p, q = j * nx + i, b * nx + a
        c = hdt * (K[j][i] + K[b][a])
        A[p][q] += c
        A[p][p] -= c
        A[q][p] += c
        A[q][q] -= c
    if bc == D:
        for j in range(ny):
            for i in range(nx):
                p = j * nx + i
                nb = sum([i == 0, i == nx - 1, j == 0, j == ny - 1])
                A[p][p] -= nb * hdt * 2 * K[j][i]
    return A


def exact_run(u0, kappa, src, steps, dt, bc):
    ny, nx = u0.shape
    hdt = Fraction(float(dt)) / 2
    A = exact_operator(kappa, bc, hdt)
    u = [Fraction(float(x)) for x in u0.reshape(-1)]
    ds = [Fraction(float(dt)) * Fraction(float(x)) for x in src.reshape(-1)]
    n = nx * ny
    for _ in range(steps):
        u = [sum((A[p][q] * u[q] for q in range(n) if A[p][q] != 0), Fraction(0)) + ds[p]
             for p in range(n)]
    return u


def dyadic_case(seed, nx=8, ny=8):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 1024, (ny, nx)) / 1024.0
    kappa = rng.integers(512, 1024, (ny, nx)) / 1024.0
    src = rng.integers(0, 1024, (ny, nx)) / 2.0 ** 20
    dt = 0.125                       # r = dt * max kappa < 0.125
    return u, kappa, src, dt


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("seed", [0, 1])
def test_brute_force_exact_first_two_steps(bc, seed):
    # With dyadic inputs the first two FP64 steps need < 53 significant bits:
    # the oracle must reproduce exact rational arithmetic bit for bit.
    u, k, s, dt = dyadic_case(seed)
    for steps in (1, 2):
        ex = np.array([float(x) for x in exact_run(u, k, s, steps, dt, bc)]).reshape(u.shape)
        got = oracle.direct(u, k, s, steps, dt, bc, "f64")
        np.testing.assert_array_equal(got, ex)


@pytest.mark.parametrize("bc", [D, P])
def test_brute_force_within_rounding_bound(bc):
    u, k, s, dt = dyadic_case(7)
    for steps in (3, 6, 10):
        ex = np.array([float(x) for x in exact_run(u, k, s, steps, dt, bc)]).reshape(u.shape)
        scale = float(np.max(np.abs(u))) + steps * dt * float(np.max(s))
        g64 = oracle.direct(u, k, s, steps, dt, bc, "f64")
        assert np.max(np.abs(g64 - ex)) <= 64 * steps * 2.0 ** -53 * scale
        g32 = oracle.direct(u.astype(np.float32), k.astype(np.float32), s.astype(np.float32),
                            steps, np.float32(dt), bc, "f32")
        assert np.max(np.abs(g32.astype(np.float64) - ex)) <= 64 * steps * 2.0 ** -24 * scale


def test_brute_force_periodic_conserves_exactly():
    u, k, _, dt = dyadic_case(3)
    s = np.zeros_like(u)
    ex = exact_run(u, k, s, 4, dt, P)
    assert sum(ex) == sum(Fraction(float(x)) for x in u.reshape(-1))


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def test_fourier_mode_decay_periodic():
    nx, ny, p, q, r, n = 64, 48, 3, 2, 0.2, 100
    kc = 0.75
    dt = r / kc
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    u0 = np.cos(2 * np.pi * (p * i / nx + q * j / ny))
    k = np.full((ny, nx), kc)
    g = 1 - 4 * r * (math.sin(math.pi * p / nx) ** 2 + math.sin(math.pi * q / ny) ** 2)
    un = oracle.direct(u0, k, np.zeros_like(u0), n, dt, P, "f64")
    assert np.max(np.abs(un - g ** n * u0)) <= 1e-12 * abs(g ** n)


def test_sine_mode_decay_dirichlet():
    nx, ny, p, q, r, n = 40, 56, 2, 5, 0.24, 100
    kc = 0.6
    dt = r / kc
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    u0 = np.sin(np.pi * p * (i + 1) / (nx + 1)) * np.sin(np.pi * q * (j + 1) / (ny + 1))
    k = np.full((ny, nx), kc)
    g = 1 - 4 * r * (math.sin(math.pi * p / (2 * (nx + 1))) ** 2
                     + math.sin(math.pi * q / (2 * (ny + 1))) ** 2)
    un = oracle.direct(u0, k, np.zeros_like(u0), n, dt, D, "f64")
    assert np.max(np.abs(un - g ** n * u0)) <= 1e-12 * abs(g ** n)


def test_conservation_periodic_fp64():
    g = W.random_grid(11, 64, 48, 1000, P, zero_source=True)
    u0 = g.u.astype(np.float64)
    un = oracle.direct(u0, g.kappa, g.src, g.steps, g.dt, P, "f64", pool=4)
    assert abs(math.fsum(un.reshape(-1)) - math.fsum(u0.reshape(-1))) <= 1e-12 * np.sum(np.abs(u0))


def test_constant_field_constant_source_periodic():
    nx, ny, n = 33, 20, 200
    u0 = np.full((ny, nx), 0.375)
    s = np.full((ny, nx), 1e-3)
    k = np.random.default_rng(2).uniform(0.5, 1.0, (ny, nx))
    dt = 0.2
    un = oracle.direct(u0, k, s, n, dt, P, "f64")
    expect = 0.375 + n * dt * 1e-3
    assert np.max(np.abs(un - expect)) <= 4 * n * 2.0 ** -53 * expect
    assert np.ptp(un) == 0.0          # every cell follows the same rounding sequence


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("bc", [D, P])
def test_maximum_principle(prec, bc):
    g = W.random_grid(5, 45, 38, 300, bc, r=0.24, zero_source=True)
    un = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, prec)
    lo = 0.0 if bc == D else float(g.u.min())      # Dirichlet ghosts are held at 0
    assert un.min() >= lo and un.max() <= float(g.u.max())


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_symmetry_bit_exact(bc, prec):
    g = W.random_grid(9, 40, 40, 25, bc)
    run = lambda u, k, s: oracle.direct(u, k, s, g.steps, g.dt, bc, prec)
    base = run(g.u, g.kappa, g.src)
    for f in (np.fliplr, np.flipud, np.transpose):
        out = run(np.ascontiguousarray(f(g.u)), np.ascontiguousarray(f(g.kappa)),
                  np.ascontiguousarray(f(g.src)))
        np.testing.assert_array_equal(out, f(base))


# ---------------------------------------------------------------------------
# fission executor == direct loop, bit for bit
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("shape,block", [((37, 29), (16, 16)), ((50, 17), (8, 4)),
                                         ((16, 16), (16, 16)), ((3, 70), (32, 2)),
                                         ((1, 1), (16, 16))])
def test_fission_equals_direct(bc, prec, shape, block):
    nx, ny = shape
    g = W.random_grid(13, nx, ny, 7, bc)
    a = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, prec)
    for pool, grain in ((1, 0), (4, 0), (3, 1), (5, 7)):
        b = oracle.fission(g.u, g.kappa, g.src, g.steps, g.dt, bc, prec, block=block, pool=pool,
                           block_per_fetch=grain)
        np.testing.assert_array_equal(a, b)


def test_direct_pool_equals_serial():
    g = W.random_grid(21, 130, 77, 9, P)
    a = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f32", pool=1)
    b = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f32", pool=6)
    np.testing.assert_array_equal(a, b)


def test_zero_steps_is_identity():
    g = W.random_grid(1, 10, 12, 0, D)
    np.testing.assert_array_equal(oracle.direct(g.u, g.kappa, g.src, 0, g.dt, D, "f32"), g.u)


# ---------------------------------------------------------------------------
# dependency-cone sampling
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_cone_sample_equals_full_run(bc, prec):
    g = W.random_grid(17, 23, 19, 13, bc)      # periodic cone wraps more than once
    full = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, bc, prec)
    idx = np.array([0, 22, 23 * 18, 23 * 19 - 1, 5 * 23 + 7, 11 * 23 + 11], np.int64)
    got = oracle.sample(g.u, g.kappa, g.src, g.steps, g.dt, bc, idx, prec)
    np.testing.assert_array_equal(got, full.reshape(-1)[idx])


# ---------------------------------------------------------------------------
# BF16
# ---------------------------------------------------------------------------
def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(100000).astype(np.float32),
        (rng.standard_normal(10000) * 1e-38).astype(np.float32),        # subnormals
        np.clip(rng.standard_normal(10000) * 3e38, -3.4e38, 3.4e38).astype(np.float32),
        np.array([0.0, -0.0, np.inf, -np.inf, 3.3895314e38, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8,
                  1.0 + 2 ** -9, 1.0 + 2 ** -8 + 2 ** -20], np.float32),
        (np.arange(65536, dtype=np.uint32) << 12 | 0x3F800000).view(np.float32),   # ties
    ])
    ours = oracle.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)


def _bf16_case(seed, nx, ny, steps, bc):
    g = W.random_grid(seed, nx, ny, steps, bc)
    st = oracle.bf16k_pack(g.u)
    kb, sb = oracle.bf16_round(g.kappa), oracle.bf16_round(g.src)
    return g, st, kb, sb


def test_bf16k_accuracy_and_stagnation_without_compensation():
    g, st, kb, sb = _bf16_case(3, 96, 80, 800, D)
    # FP64 reference on the bf16-quantised inputs isolates the storage error.
    k64, s64 = oracle.bf16_to_f32(kb).astype(np.float64), oracle.bf16_to_f32(sb).astype(np.float64)
    ref = oracle.direct(oracle.bf16k_value(st), k64, s64, g.steps, g.dt, D, "f64")
    comp = oracle.bf16k_value(oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, D))
    plain = oracle.bf16k_value(oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, D, compensate=False))
    err_c = np.max(np.abs(comp - ref)) / np.max(np.abs(ref))
    err_p = np.max(np.abs(plain - ref)) / np.max(np.abs(ref))
    assert err_c <= 1e-3
    assert err_p > 10 * err_c          # without compensation small increments are lost


def test_bf16k_pool_equals_serial():
    g, st, kb, sb = _bf16_case(4, 70, 33, 11, P)
    a = oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, P, pool=1)
    b = oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, P, pool=5)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("bc", [D, P])
def test_bf16k_block_with_depth_one_passes_is_per_step_rounding(bc):
    # Rounding once per pass with passes of one step is rounding every step:
    # the Python composition (FP32 loop + pack) equals the C++ BF16-Kahan loop.
    for seed, nx, ny, steps in ((5, 70, 33, 11), (6, 9, 130, 7), (7, 1, 1, 3)):
        g, st, kb, sb = _bf16_case(seed, nx, ny, steps, bc)
        a = oracle.direct_bf16k(st, kb, sb, steps, g.dt, bc)
        b = oracle.direct_bf16k_block(st, kb, sb, [1] * steps, g.dt, bc)
        np.testing.assert_array_equal(a, b)


def test_bf16k_block_accuracy():
    # Rounded once per pass of 8 steps, the storage error against FP64 on the
    # bf16-quantised inputs is no larger than with every step rounded.
    g, st, kb, sb = _bf16_case(3, 96, 80, 800, D)
    k64, s64 = oracle.bf16_to_f32(kb).astype(np.float64), oracle.bf16_to_f32(sb).astype(np.float64)
    ref = oracle.direct(oracle.bf16k_value(st), k64, s64, g.steps, g.dt, D, "f64")
    every = oracle.bf16k_value(oracle.direct_bf16k(st, kb, sb, g.steps, g.dt, D))
    block = oracle.bf16k_value(oracle.direct_bf16k_block(st, kb, sb, oracle.pass_schedule(g.steps, 8), g.dt, D))
    err_e = np.max(np.abs(every - ref)) / np.max(np.abs(ref))
    err_b = np.max(np.abs(block - ref)) / np.max(np.abs(ref))
    assert err_b <= err_e and err_b <= 1e-3


def test_pass_schedule():
    for steps in range(0, 40):
        for k in range(1, 9):
            for scratch in (True, False):
                d = oracle.pass_schedule(steps, k, scratch)
                assert sum(d) == steps and all(1 <= x <= k for x in d)
                if not scratch and any(x >= 2 for x in d):
                    assert len(d) % 2 == 1
    assert oracle.pass_schedule(17, 4) == [4, 4, 4, 4, 1]
    assert oracle.pass_schedule(16, 4, False) == [4, 4, 4, 2, 2]
    assert oracle.pass_schedule(9, 4, False) == [4, 4, 1]


def test_bf16k_pack_represents_float_closely():
    u = np.random.default_rng(1).random(10000, dtype=np.float32)
    v = oracle.bf16k_value(oracle.bf16k_pack(u))
    assert np.max(np.abs(v - u.astype(np.float64)) / u.astype(np.float64).clip(1e-6)) < 2 ** -16


# ---------------------------------------------------------------------------
# heat sum
# ---------------------------------------------------------------------------
def test_heat_sum_within_order_bound():
    u = np.random.default_rng(3).random(1 << 20, dtype=np.float32)
    exact = math.fsum(u.astype(np.float64))
    got = oracle.heat_sum_f32(u)
    assert abs(got - exact) <= u.size * 2.0 ** -52 * float(u.max())
    st = oracle.bf16k_pack(u[:4096])
    exact_b = math.fsum(oracle.bf16k_value(st))
    assert abs(oracle.heat_sum_bf16k(st) - exact_b) <= 4096 * 2.0 ** -52


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
def _loss(u0, k, s, target, steps, dt, bc):
    uT = oracle.direct(u0, k, s, steps, dt, bc, "f64")
    return 0.5 * math.fsum(((uT - target) ** 2).reshape(-1))


@pytest.mark.parametrize("bc", [D, P])
def test_adjoint_against_central_differences(bc):
    nx, ny, steps, ckpt = 24, 20, 30, 7
    g = W.differentiation(seed=5, n=nx, ny=ny, steps=steps, ckpt=ckpt)
    u0, k = g.u.astype(np.float64), g.kappa.astype(np.float64)
    s = np.zeros_like(u0)
    tgt = g.extras["target"].astype(np.float64)
    L, gu, gk = oracle.adjoint_f64(u0, k, s, tgt, steps, float(g.dt), bc, ckpt)
    assert abs(L - _loss(u0, k, s, tgt, steps, float(g.dt), bc)) <= 1e-12 * L
    eps = 1e-3
    for d in W.unit_directions(6, 8, u0.shape):
        # L is quadratic in u0: the central difference is exact up to rounding.
        fd = (_loss(u0 + eps * d, k, s, tgt, steps, g.dt, bc)
              - _loss(u0 - eps * d, k, s, tgt, steps, g.dt, bc)) / (2 * eps)
        gd = float(np.sum(gu * d))
        assert abs(fd - gd) <= 1e-6 * abs(gd) + 1e-10
        fd = (_loss(u0, k + eps * d, s, tgt, steps, g.dt, bc)
              - _loss(u0, k - eps * d, s, tgt, steps, g.dt, bc)) / (2 * eps)
        gd = float(np.sum(gk * d))
        assert abs(fd - gd) <= 1e-6 * abs(gd) + 1e-10


def test_adjoint_64_directions_on_the_differentiation_schedule():
    # The differentiation workload's schedule and fields (Dirichlet, kappa ~
    # U[0.5, 1), u0 ~ U[0, 1), no source, r = 0.2, 200 steps, checkpoints every
    # 20, target = 8 seeded sinusoids) on a 128 x 128 grid: the FP64 adjoint
    # against FP64 central differences (eps = 1e-3) on 64 seeded unit
    # directions each for u0 and kappa.
    g = W.differentiation(seed=4, n=128, steps=200, ckpt=20)
    u0, k = g.u.astype(np.float64), g.kappa.astype(np.float64)
    s = np.zeros_like(u0)
    tgt = g.extras["target"].astype(np.float64)
    steps, ckpt, dt = g.steps, g.extras["ckpt"], float(g.dt)
    L, gu, gk = oracle.adjoint_f64(u0, k, s, tgt, steps, dt, g.bc, ckpt, pool=4)
    assert abs(L - _loss(u0, k, s, tgt, steps, dt, g.bc)) <= 1e-12 * L
    eps = 1e-3
    for d in W.unit_directions(40, 64, u0.shape):
        fd = (_loss(u0 + eps * d, k, s, tgt, steps, dt, g.bc)
              - _loss(u0 - eps * d, k, s, tgt, steps, dt, g.bc)) / (2 * eps)
        gd = float(np.sum(gu * d))
        assert abs(fd - gd) <= 1e-6 * abs(gd) + 1e-10
        fd = (_loss(u0, k + eps * d, s, tgt, steps, dt, g.bc)
              - _loss(u0, k - eps * d, s, tgt, steps, dt, g.bc)) / (2 * eps)
        gd = float(np.sum(gk * d))
        assert abs(fd - gd) <= 1e-6 * abs(gd) + 1e-10


def test_adjoint_checkpoint_interval_does_not_change_result():
    g = W.differentiation(seed=8, n=17, ny=13, steps=23)
    u0, k = g.u.astype(np.float64), g.kappa.astype(np.float64)
    s = np.zeros_like(u0)
    tgt = g.extras["target"].astype(np.float64)
    ref = oracle.adjoint_f64(u0, k, s, tgt, 23, float(g.dt), D, 1)
    for ck in (4, 23, 50):
        out = oracle.adjoint_f64(u0, k, s, tgt, 23, float(g.dt), D, ck)
        assert out[0] == ref[0]
        np.testing.assert_array_equal(out[1], ref[1])
        np.testing.assert_array_equal(out[2], ref[2])


def test_adjoint_with_source_matches_fd():
    # A source enters only additively: the gradient is unchanged in form.
    nx, ny, steps = 12, 10, 15
    g = W.random_grid(31, nx, ny, steps, D)
    u0, k, s = (x.astype(np.float64) for x in (g.u, g.kappa, g.src))
    tgt = np.zeros_like(u0)
    _, gu, gk = oracle.adjoint_f64(u0, k, s, tgt, steps, float(g.dt), D, 4)
    d = W.unit_directions(2, 1, u0.shape)[0]
    eps = 1e-3
    fd = (_loss(u0, k + eps * d, s, tgt, steps, g.dt, D)
          - _loss(u0, k - eps * d, s, tgt, steps, g.dt, D)) / (2 * eps)
    assert abs(fd - float(np.sum(gk * d))) <= 1e-6 * abs(fd) + 1e-10
