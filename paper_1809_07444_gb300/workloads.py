"""Seeded synthetic inputs for the SMMO applications.

These generators produce the starting states that both the CUDA path and the
oracle take as inputs. They hold none of the method's arithmetic: no
allocation, no do-all and no application rule is computed here, only the
initial grids, bodies, instance sizes and job streams, drawn from numpy's
PCG64 generator (platform independent) with an explicit seed.

Shapes and distributions follow the workloads the applications run on:
  - game of life: W x H torus, each cell alive with probability 0.25;
  - wa-tor: W x H torus, 30% of the cells hold a fish and 3% a shark, the rest
    are empty;
  - n-body: positions uniform in the unit cube, masses log-uniform in
    [1e-3, 1], zero velocity, values rounded to float32 so that the FP32 GPU
    state and the FP64 oracle start from the same numbers; a draw is rejected
    (and the seed advanced) while some pair lies within `margin` of the merge
    distance;
  - traffic: R roads of L cells, each cell holds a car with probability
    `density`, with a velocity uniform in {0, ..., vmax};
  - sugarscape: W x H torus with two sugar hills (capacity 4 at the peaks,
    (W/4, H/4) and (3W/4, 3H/4), falling by 1 every W/10 cells of distance,
    floor at 0); each cell holds an agent with probability `density`, with
    sugar uniform in [5, 25], metabolism in [1, 4], vision in [1, 6],
    maximum age in [60, 100] and an age uniform below it;
  - batched wa-tor: side lengths log-uniform in [64, 1024];
  - served jobs: Poisson arrivals, game-of-life or wa-tor with equal odds,
    sides log-uniform in [128, 4096], step counts uniform in [50, 1000].
"""
import numpy as np

EMPTY, FISH, SHARK = 0, 1, 2


def gol_initial(W, H, seed, density=0.25):
    """uint8[H, W]: 1 where the cell starts alive."""
    rng = np.random.default_rng(seed)
    return (rng.random((H, W)) < density).astype(np.uint8)


def wator_initial(W, H, seed, fish=0.30, shark=0.03):
    """uint8[H, W] of EMPTY / FISH / SHARK."""
    rng = np.random.default_rng(seed)
    u = rng.random((H, W))
    k = np.zeros((H, W), dtype=np.uint8)
    k[u < fish] = FISH
    k[(u >= fish) & (u < fish + shark)] = SHARK
    return k


def traffic_initial(R, L, seed, density=0.2, vmax=5):
    """int8[R, L]: -1 for an empty cell, else the initial velocity of its car."""
    rng = np.random.default_rng(seed)
    occupied = rng.random((R, L)) < density
    v = rng.integers(0, vmax + 1, size=(R, L))
    return np.where(occupied, v, -1).astype(np.int8)


def sugarscape_initial(W, H, seed, density=0.1):
    """(cap uint8[H, W], agents int32[n, 7] = x, y, sugar, metabolism,
    vision, age, max_age)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    step = max(W, H) / 10.0
    cap = np.zeros((H, W), dtype=np.int64)
    for px, py in ((W / 4, H / 4), (3 * W / 4, 3 * H / 4)):
        dx = np.minimum(np.abs(x - px), W - np.abs(x - px))
        dy = np.minimum(np.abs(y - py), H - np.abs(y - py))
        cap = np.maximum(cap, 4 - np.floor(np.hypot(dx, dy) / step).astype(np.int64))
    cap = np.clip(cap, 0, 4).astype(np.uint8)
    cells = np.flatnonzero(rng.random(W * H) < density)
    n = len(cells)
    max_age = rng.integers(60, 101, n)
    agents = np.stack([cells % W, cells // W, rng.integers(5, 26, n), rng.integers(1, 5, n), rng.integers(1, 7, n),
                       (rng.random(n) * max_age).astype(np.int64), max_age], 1).astype(np.int32)
    return cap, agents


def nbody_initial(n, seed, r_merge=2e-3, margin=1e-5, max_tries=64):
    """(float64[n, 7] rows (x, y, z, vx, vy, vz, m), seed actually used).

    All values are exactly representable in float32.
    """
    from scipy.spatial import cKDTree

    for k in range(max_tries):
        rng = np.random.default_rng(seed + k)
        pos = rng.random((n, 3)).astype(np.float32).astype(np.float64)
        m = (10.0 ** rng.uniform(-3.0, 0.0, n)).astype(np.float32).astype(np.float64)
        if margin > 0 and n > 1:
            tree = cKDTree(pos)
            pairs = tree.query_pairs(r_merge + margin, output_type="ndarray")
            if len(pairs):
                d = np.linalg.norm(pos[pairs[:, 0]] - pos[pairs[:, 1]], axis=1)
                if np.any(np.abs(d - r_merge) < margin):
                    continue
        rows = np.zeros((n, 7), dtype=np.float64)
        rows[:, 0:3] = pos
        rows[:, 6] = m
        return rows, seed + k
    raise RuntimeError("no admissible n-body draw within max_tries seeds")


def batched_sides(n, seed, lo=64, hi=1024):
    """int64[n] side lengths, floor(exp(U[ln lo, ln hi]))."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), n))).astype(np.int64)


def served_jobs(n, seed, rate=200.0, lo=128, hi=4096, steps_lo=50, steps_hi=1000):
    """Job stream as a dict of arrays: arrival (s), app (0 = life, 1 = wa-tor), side, steps, seed."""
    rng = np.random.default_rng(seed)
    arrival = np.cumsum(rng.exponential(1.0 / rate, n))
    app = (rng.random(n) < 0.5).astype(np.int64)
    side = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), n))).astype(np.int64)
    steps = rng.integers(steps_lo, steps_hi + 1, n)
    seeds = rng.integers(0, 2**31 - 1, n)
    return {"arrival": arrival, "app": app, "side": side, "steps": steps, "seed": seeds}
