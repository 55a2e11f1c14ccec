"""Pins for the oracle's 3-D 7-point variant (the paper's hotspot3D class).

Update (a stated reading: the 2-D flux-form step with a third pair of faces):
acc = ((fW + fE) + (fS + fN)) + (fD + fU), u' = c + (hdt * acc + dt * s),
f = (kc + kn)(un - c), hdt = dt / 2; Dirichlet ghosts u = 0, kappa = kc;
periodic wraps.  Pinned against exact rational arithmetic through an operator
assembled face by face, closed-form decay factors, exact conservation, the
maximum principle, bit-exact symmetries, the 2-D update (nz = 1, periodic),
and the z-marching tiled kernel executed with loop fission.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

D, P = W.DIRICHLET, W.PERIODIC


def exact_run3(u0, kappa, src, steps, dt, bc):
    """Exact Fractions: per face (p, q) with conductivity hdt (k_p + k_q) heat
    moves from the hotter to the colder cell; a Dirichlet boundary face of p
    conducts hdt (2 k_p) towards a ghost at zero."""
    nz, ny, nx = u0.shape
    n = nx * ny * nz
    idx = lambda i, j, k: (k * ny + j) * nx + i  # noqa: E731
    K = [Fraction(float(x)) for x in kappa.reshape(-1)]
    hdt = Fraction(float(dt)) / 2
    faces, bnd = [], [0] * n
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = idx(i, j, k)
                for axis, m in ((0, nx), (1, ny), (2, nz)):
                    q = [i, j, k]
                    q[axis] += 1
                    if q[axis] < m:
                        faces.append((p, idx(*q)))
                    elif bc == P:
                        q[axis] = 0
                        faces.append((p, idx(*q)))
                    else:
                        bnd[p] += 1
                    if bc == D and [i, j, k][axis] == 0:
                        bnd[p] += 1
    u = [Fraction(float(x)) for x in u0.reshape(-1)]
    ds = [Fraction(float(dt)) * Fraction(float(x)) for x in src.reshape(-1)]
    for _ in range(steps):
        nu = list(u)
        for p, q in faces:
            flow = hdt * (K[p] + K[q]) * (u[q] - u[p])
            nu[p] += flow
            nu[q] -= flow
        for p in range(n):
            nu[p] += -bnd[p] * hdt * 2 * K[p] * u[p] + ds[p]
        u = nu
    return np.array([float(x) for x in u]).reshape(u0.shape), u


def dyadic3(seed, shape=(3, 4, 5)):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 1024, shape) / 1024.0
    k = rng.integers(512, 1024, shape) / 1024.0
    s = rng.integers(0, 1024, shape) / 2.0 ** 20
    return u, k, s, 0.125


@pytest.mark.parametrize("bc", [D, P])
def test_exact_first_two_steps_3d(bc):
    u, k, s, dt = dyadic3(0)
    for steps in (1, 2):
        ex, _ = exact_run3(u, k, s, steps, dt, bc)
        np.testing.assert_array_equal(oracle.direct3(u, k, s, steps, dt, bc, "f64"), ex)


@pytest.mark.parametrize("bc", [D, P])
def test_within_rounding_bound_3d(bc):
    u, k, s, dt = dyadic3(3, (4, 3, 6))
    for steps in (4, 8):
        ex, _ = exact_run3(u, k, s, steps, dt, bc)
        scale = 1.0 + steps * dt * float(np.max(s))
        g64 = oracle.direct3(u, k, s, steps, dt, bc, "f64")
        assert np.max(np.abs(g64 - ex)) <= 64 * steps * 2.0 ** -53 * scale
        g32 = oracle.direct3(*(x.astype(np.float32) for x in (u, k, s)), steps, np.float32(dt), bc, "f32")
        assert np.max(np.abs(g32.astype(np.float64) - ex)) <= 64 * steps * 2.0 ** -24 * scale


def test_periodic_conserves_exactly_in_rational_arithmetic_3d():
    u, k, _, dt = dyadic3(5)
    _, ex = exact_run3(u, k, np.zeros_like(u), 6, dt, P)
    assert sum(ex) == sum(Fraction(float(x)) for x in u.reshape(-1))


def test_periodic_fourier_mode_decay_3d():
    nx, ny, nz, p, q, w, kap, r, steps = 16, 12, 10, 2, 1, 3, 0.75, 0.15, 60
    dt = r / kap
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="xy")
    i, j, k = (np.transpose(a, (2, 0, 1)) for a in (i, j, k))
    u0 = np.cos(2 * np.pi * (p * i / nx + q * j / ny + w * k / nz))
    g = 1 - 4 * r * (math.sin(math.pi * p / nx) ** 2 + math.sin(math.pi * q / ny) ** 2
                     + math.sin(math.pi * w / nz) ** 2)
    got = oracle.direct3(u0, np.full(u0.shape, kap), np.zeros(u0.shape), steps, dt, P, "f64")
    # error relative to the initial amplitude 1 (rounding leaves ~1e-17 in the
    # constant mode, which never decays)
    np.testing.assert_allclose(got, g ** steps * u0, rtol=0, atol=1e-12)


def test_dirichlet_sine_mode_decay_3d():
    nx, ny, nz, p, q, w, kap, r, steps = 9, 7, 6, 2, 3, 1, 0.6, 0.15, 50
    dt = r / kap
    k3, j3, i3 = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u0 = (np.sin(np.pi * p * (i3 + 1) / (nx + 1)) * np.sin(np.pi * q * (j3 + 1) / (ny + 1))
          * np.sin(np.pi * w * (k3 + 1) / (nz + 1)))
    g = 1 - 4 * r * (math.sin(math.pi * p / (2 * (nx + 1))) ** 2 + math.sin(math.pi * q / (2 * (ny + 1))) ** 2
                     + math.sin(math.pi * w / (2 * (nz + 1))) ** 2)
    got = oracle.direct3(u0, np.full(u0.shape, kap), np.zeros(u0.shape), steps, dt, D, "f64")
    np.testing.assert_allclose(got, g ** steps * u0, rtol=0, atol=1e-12)


def test_conservation_drift_fp64_3d():
    g = W.random_grid3(9, 24, 20, 16, 400, P, zero_source=True)
    u, k = g.u.astype(np.float64), g.kappa.astype(np.float64)
    out = oracle.direct3(u, k, np.zeros_like(u), g.steps, float(g.dt), P, "f64", pool=4)
    assert abs(math.fsum(out.reshape(-1)) - math.fsum(u.reshape(-1))) <= 1e-12 * math.fsum(np.abs(u).reshape(-1))


@pytest.mark.parametrize("bc", [D, P])
def test_max_principle_3d(bc):
    g = W.random_grid3(10, 17, 13, 11, 40, bc, zero_source=True)
    out = oracle.direct3(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
    lo = 0.0 if bc == D else float(g.u.min())
    assert out.min() >= lo and out.max() <= g.u.max()


@pytest.mark.parametrize("bc", [D, P])
def test_mirror_and_xy_transpose_symmetry_bit_exact_3d(bc):
    g = W.random_grid3(11, 14, 14, 9, 7, bc)
    ref = oracle.direct3(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
    for ax in (0, 1, 2):
        f = lambda a: np.ascontiguousarray(np.flip(a, ax))  # noqa: E731
        got = oracle.direct3(f(g.u), f(g.kappa), f(g.src), g.steps, g.dt, bc, "f32")
        np.testing.assert_array_equal(got, f(ref))
    t = lambda a: np.ascontiguousarray(np.transpose(a, (0, 2, 1)))  # noqa: E731
    got = oracle.direct3(t(g.u), t(g.kappa), t(g.src), g.steps, g.dt, bc, "f32")
    np.testing.assert_array_equal(got, t(ref))


def test_single_periodic_plane_is_the_2d_update():
    # nz = 1, periodic: the z neighbours are the cell itself, fD = fU = 0 and
    # acc = (2-D acc) + 0 exactly.
    g = W.random_grid(12, 37, 23, 9, P)
    ref = oracle.direct(g.u, g.kappa, g.src, g.steps, g.dt, P, "f32")
    got = oracle.direct3(g.u[None], g.kappa[None], g.src[None], g.steps, g.dt, P, "f32")
    np.testing.assert_array_equal(got[0], ref)


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("shape,block,zc", [((21, 13, 9), (8, 4), 3), ((40, 33, 17), (32, 8), 1),
                                            ((5, 3, 2), (16, 16), 4), ((1, 1, 1), (32, 8), 1),
                                            ((64, 8, 30), (32, 2), 7)])
def test_fission3_equals_direct3(bc, shape, block, zc):
    nx, ny, nz = shape
    g = W.random_grid3(13, nx, ny, nz, 5, bc)
    ref = oracle.direct3(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32")
    got = oracle.fission3(g.u, g.kappa, g.src, g.steps, g.dt, bc, "f32", block=block, zchunks=zc, pool=3)
    np.testing.assert_array_equal(got, ref)
    u, k, s = (x.astype(np.float64) for x in (g.u, g.kappa, g.src))
    np.testing.assert_array_equal(
        oracle.fission3(u, k, s, 3, float(g.dt), bc, "f64", block=block, zchunks=zc, pool=2),
        oracle.direct3(u, k, s, 3, float(g.dt), bc, "f64"))
