"""Slab decomposition of the 2-D heat stencil across ranks, with halo exchange.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only tests/ import it.
It shares no code with the CUDA library.

The multi-GPU plan of the stencil: rank r of R owns a contiguous block of
rows [lo, hi) of the ny x nx grid (full width).  It keeps H = K halo rows
above and below its own rows.  Every K steps it exchanges H rows of u with
each neighbouring rank, then advances up to K steps locally.  Step t of such
a block is valid on local rows [t, n + 2H - t), so after K steps the own rows
are exact again.

Boundaries:
* Periodic y: the ranks form a ring, so rank 0's lower neighbour is rank R-1.
  With one rank the halos are the rank's own wrapped rows (a local copy).
* Dirichlet y: the rows past the grid edge are ghosts.  They hold u = 0 at
  every step, and κ of the in-grid row they touch (a boundary face conducts
  with 2 κ_c).  Nothing is exchanged past the edge.

κ and s never change, so their halos are exchanged once, at the start.  The
per-cell update is the flux form in the canonical rounding order, every
operation in the working precision:
    fW = (kc + kW)(uW - c),  fE, fS, fN alike,
    acc = (fW + fE) + (fS + fN),
    u' = c + (hdt * acc + dt * s),   hdt = 0.5 * dt.
It is written out with numpy elementwise operations, which round each
operation in the array's precision (no contraction).

A rank must own at least K rows, so that its halos come from its immediate
neighbours only.
"""
from __future__ import annotations

import numpy as np

DIRICHLET = 0
PERIODIC = 1


def split_rows(ny: int, world: int) -> list[tuple[int, int]]:
    """Contiguous row ranges [lo, hi) of `world` ranks; the sizes differ by at most one."""
    if world < 1 or ny < world:
        raise ValueError(f"cannot split {ny} rows over {world} ranks")
    base, extra = divmod(ny, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


class LocalExchange:
    """One rank, periodic: the lower halo is the rank's own last rows and the upper halo its first rows."""

    def __init__(self, periodic: bool):
        self.periodic = periodic

    def swap(self, to_lower: np.ndarray, to_upper: np.ndarray):
        """Send `to_lower` to the lower neighbour and `to_upper` to the upper one;
        return (from_lower, from_upper), or None for a side without a neighbour."""
        if not self.periodic:
            return None, None
        return to_upper.copy(), to_lower.copy()


class TorchDistExchange:
    """Neighbour exchange over torch.distributed point-to-point messages (gloo on CPU)."""

    TAG_UP, TAG_DOWN = 11, 12

    def __init__(self, rank: int, world: int, periodic: bool, skip_after: int | None = None):
        self.rank, self.world, self.periodic = rank, world, periodic
        self.lower = (rank - 1) % world if (periodic or rank > 0) else None
        self.upper = (rank + 1) % world if (periodic or rank < world - 1) else None
        # Tests only: after this many swaps, return stale halos without communicating.
        self.skip_after = skip_after
        self.calls = 0
        self._last = (None, None)

    def swap(self, to_lower: np.ndarray, to_upper: np.ndarray):
        import torch
        import torch.distributed as dist

        self.calls += 1
        if self.skip_after is not None and self.calls > self.skip_after:
            return self._last
        reqs, got_lower, got_upper = [], None, None
        if self.lower is not None:
            got_lower = torch.empty(to_upper.shape, dtype=torch.from_numpy(to_upper).dtype)
            reqs.append(dist.irecv(got_lower, src=self.lower, tag=self.TAG_UP))
        if self.upper is not None:
            got_upper = torch.empty(to_lower.shape, dtype=torch.from_numpy(to_lower).dtype)
            reqs.append(dist.irecv(got_upper, src=self.upper, tag=self.TAG_DOWN))
        if self.upper is not None:  # my top rows are my upper neighbour's lower halo
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(to_upper)), dst=self.upper,
                                   tag=self.TAG_UP))
        if self.lower is not None:  # my bottom rows are my lower neighbour's upper halo
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(to_lower)), dst=self.lower,
                                   tag=self.TAG_DOWN))
        for q in reqs:
            q.wait()
        self._last = (None if got_lower is None else got_lower.numpy().copy(),
                      None if got_upper is None else got_upper.numpy().copy())
        return self._last


class ThreadExchange:
    """Ranks as threads of one process; each rank has a mailbox per direction.

    ``make(world, periodic)`` returns one exchange object per rank; run each
    rank's ``run_slab`` on its own thread."""

    def __init__(self, rank, world, periodic, boxes):
        self.rank, self.world = rank, world
        self.lower = (rank - 1) % world if (periodic or rank > 0) else None
        self.upper = (rank + 1) % world if (periodic or rank < world - 1) else None
        self.boxes = boxes  # boxes[(dst, direction)]: "up" = sent by the rank below, "down" = by the rank above

    @staticmethod
    def make(world, periodic):
        import queue
        boxes = {(r, d): queue.Queue() for r in range(world) for d in ("up", "down")}
        return [ThreadExchange(r, world, periodic, boxes) for r in range(world)]

    def swap(self, to_lower, to_upper, timeout=60.0):
        if self.upper is not None:
            self.boxes[(self.upper, "up")].put(np.array(to_upper, copy=True))
        if self.lower is not None:
            self.boxes[(self.lower, "down")].put(np.array(to_lower, copy=True))
        got_lower = self.boxes[(self.rank, "up")].get(timeout=timeout) if self.lower is not None else None
        got_upper = self.boxes[(self.rank, "down")].get(timeout=timeout) if self.upper is not None else None
        return got_lower, got_upper


def run_threads(u, kappa, src, steps, dt, bc, K, world, precision="f32"):
    """All ranks of the decomposition as threads; returns the assembled result."""
    import threading
    ex = ThreadExchange.make(world, bc == PERIODIC)
    out, err = [None] * world, []

    def rank_main(r):
        try:
            out[r] = run_slab(u, kappa, src, steps, dt, bc, K, r, world, ex[r], precision)
        except Exception as e:  # reported to the caller below
            err.append(e)

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    return np.concatenate(out, axis=0)


def _step_rows(U, Kp, S, r0, r1, periodic_x, dt, hdt):
    """Return the updated rows [r0, r1) of the local arrays (one step, canonical order)."""
    c, kc = U[r0:r1], Kp[r0:r1]
    uS, kS = U[r0 - 1:r1 - 1], Kp[r0 - 1:r1 - 1]
    uN, kN = U[r0 + 1:r1 + 1], Kp[r0 + 1:r1 + 1]
    if periodic_x:
        uW, kW = np.roll(c, 1, axis=1), np.roll(kc, 1, axis=1)
        uE, kE = np.roll(c, -1, axis=1), np.roll(kc, -1, axis=1)
    else:  # Dirichlet x: ghost u = 0, ghost κ = κ_c
        zero = np.zeros((c.shape[0], 1), c.dtype)
        uW = np.concatenate([zero, c[:, :-1]], axis=1)
        uE = np.concatenate([c[:, 1:], zero], axis=1)
        kW = np.concatenate([kc[:, :1], kc[:, :-1]], axis=1)
        kE = np.concatenate([kc[:, 1:], kc[:, -1:]], axis=1)
    fW = (kc + kW) * (uW - c)
    fE = (kc + kE) * (uE - c)
    fS = (kc + kS) * (uS - c)
    fN = (kc + kN) * (uN - c)
    acc = (fW + fE) + (fS + fN)
    return c + (hdt * acc + dt * S[r0:r1])


def run_slab(u, kappa, src, steps, dt, bc, K, rank, world, exchange, precision="f32"):
    """Advance rank `rank`'s slab of the grid by `steps` steps; returns its own rows.

    u, kappa, src: the full (ny, nx) input fields.  The rank reads only its own
    rows of them; every halo row reaches it through `exchange`.  bc applies
    to both axes, as in the single-grid stencil."""
    ft = np.float64 if precision == "f64" else np.float32
    ny, nx = u.shape
    lo, hi = split_rows(ny, world)[rank]
    n, H = hi - lo, K
    if K < 1:
        raise ValueError("K must be >= 1")
    if world > 1 and min(b - a for a, b in split_rows(ny, world)) < K:
        raise ValueError(f"every rank needs at least K = {K} rows")
    if world == 1 and bc == PERIODIC and n < K:
        raise ValueError(f"a periodic single rank needs at least K = {K} rows")
    periodic = bc == PERIODIC
    dt = ft(dt)
    hdt = ft(0.5) * dt

    U = np.zeros((n + 2 * H, nx), ft)
    Kp = np.zeros((n + 2 * H, nx), ft)
    S = np.zeros((n + 2 * H, nx), ft)
    U[H:H + n] = u[lo:hi]
    Kp[H:H + n] = kappa[lo:hi]
    S[H:H + n] = src[lo:hi]

    # Global row of each local row; rows outside [0, ny) are Dirichlet ghosts.
    grow = np.arange(lo - H, hi + H)
    inside = (grow >= 0) & (grow < ny) if not periodic else np.ones_like(grow, bool)

    def fill_halos(A, got_lower, got_upper, ghost_lower, ghost_upper):
        if got_lower is not None:
            A[:H] = got_lower
        else:
            A[:H] = ghost_lower
        if got_upper is not None:
            A[H + n:] = got_upper
        else:
            A[H + n:] = ghost_upper

    # Static halos of κ and s, once.  Dirichlet ghost rows take κ of the edge row.
    kl, ku = exchange.swap(Kp[H:2 * H].copy(), Kp[n:n + H].copy())
    fill_halos(Kp, kl, ku, np.broadcast_to(Kp[H], (H, nx)), np.broadcast_to(Kp[H + n - 1], (H, nx)))
    sl, su = exchange.swap(S[H:2 * H].copy(), S[n:n + H].copy())
    fill_halos(S, sl, su, 0, 0)

    done = 0
    while done < steps:
        k = min(K, steps - done)
        ul, uu = exchange.swap(U[H:2 * H].copy(), U[n:n + H].copy())
        fill_halos(U, ul, uu, 0, 0)
        for t in range(1, k + 1):
            r0, r1 = t, n + 2 * H - t
            new = _step_rows(U, Kp, S, r0, r1, periodic, dt, hdt)
            keep = inside[r0:r1]
            U[r0:r1][keep] = new[keep]  # Dirichlet ghost rows stay at u = 0
        done += k
    return U[H:H + n].copy()
