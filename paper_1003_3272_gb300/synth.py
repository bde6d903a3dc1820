"""Seeded synthetic inputs for the NMF workloads.

This module is the one piece of code shared by the CUDA path, the FP64 oracle,
the tests and the benchmark: it only *draws numbers*.  It contains none of the
multiplicative-update arithmetic.

Generator: a counter-based SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Word ``i`` of stream ``s`` under
seed ``seed`` is

    key  = mix64(seed + (s + 1) * GAMMA)          (mod 2**64)
    word = mix64(key  + (i + 1) * GAMMA)          (mod 2**64)

with GAMMA = 0x9E3779B97F4A7C15 and the SplitMix64 finaliser

    mix64(z): z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
              z = (z ^ (z >> 27)) * 0x94D049BB133111EB
              return z ^ (z >> 31)

Distributions (all produced in float32 unless stated):
  * uniform on [0,1):   (word >> 40) * 2**-24                 exact in fp32
  * uniform on (0,1):   ((word >> 41) + 0.5) * 2**-23         exact, never 0 or 1
  * Exponential(1) = Gamma(1,1):  -log(((word >> 11) + 0.5) * 2**-53) in fp64,
    rounded once to fp32
  * |N(0, sigma^2)|:  Box-Muller on words 2i (radius) and 2i+1 (angle), fp64,
    rounded once to fp32

The CUDA library's seeded initialisation of W and H (Algorithm 1's "draw
uniform on (0,1)") implements the same uniform-(0,1) definition on the device;
a test checks the two bit for bit.

Workloads: the five problem families the method is measured on (a CBCL-shaped
faces matrix, a planted low-rank matrix, a tall uniform matrix for the
precision sweep, a batch of small uneven problems and a large streaming
matrix).  Each builder returns V together with the seeded starting factors.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids: the data matrix, the left and right starting factors, and the
# planted factors / noise of the planted workload.
STREAM_V = 0
STREAM_W = 1
STREAM_H = 2
STREAM_WSTAR = 3
STREAM_HSTAR = 4
STREAM_NOISE = 5
STREAM_SHAPES = 6
STREAM_COUNTS = 7
STREAM_PET_COUNTS = 8

BASE_SEED = 20100316


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        z = np.array([seed % (1 << 64)], dtype=np.uint64)
        z = z + np.uint64(stream + 1) * GAMMA
        return _mix64(z)[0]


def words(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Raw 64-bit words ``start .. start+count-1`` of one stream."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(key + idx * GAMMA)


_CHUNK = 1 << 22


def _chunks(count, body):
    """Run ``body(start, length)`` over chunks of ``count``; large fills use a
    thread pool (numpy releases the GIL inside the array operations).  The
    chunks write disjoint slices, so the result does not depend on the
    schedule."""
    starts = range(0, count, _CHUNK)
    if count <= 4 * _CHUNK:
        for s in starts:
            body(s, min(_CHUNK, count - s))
        return
    import concurrent.futures as cf
    import os
    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        list(ex.map(lambda s: body(s, min(_CHUNK, count - s)), starts))


def _fill(seed, stream, count, fn, dtype=np.float32):
    out = np.empty(count, dtype=dtype)

    def body(s, c):
        out[s:s + c] = fn(words(seed, stream, s, c))
    _chunks(count, body)
    return out


def uniform_open(seed: int, stream: int, shape) -> np.ndarray:
    """iid uniform on (0,1), float32, row-major ``shape``."""
    n = int(np.prod(shape))
    f = lambda w: ((w >> np.uint64(41)).astype(np.float64) + 0.5) * 2.0 ** -23
    return _fill(seed, stream, n, f).reshape(shape)


def uniform_closed_open(seed: int, stream: int, shape) -> np.ndarray:
    """iid uniform on [0,1), float32."""
    n = int(np.prod(shape))
    f = lambda w: (w >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    return _fill(seed, stream, n, f).reshape(shape)


def exponential(seed: int, stream: int, shape) -> np.ndarray:
    """iid Exponential(1) (= Gamma(1,1)), float32."""
    n = int(np.prod(shape))
    f = lambda w: -np.log(((w >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53)
    return _fill(seed, stream, n, f).reshape(shape)


def abs_normal(seed: int, stream: int, shape, sigma: float) -> np.ndarray:
    """iid |N(0, sigma^2)|, float32 (Box-Muller over word pairs)."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float32)

    def body(s, c):
        w = words(seed, stream, 2 * s, 2 * c)
        u1 = ((w[0::2] >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        u2 = ((w[1::2] >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        out[s:s + c] = np.abs(sigma * z)
    _chunks(n, body)
    return out.reshape(shape)


def uniform_int(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """iid integers uniform on {lo..hi} (inclusive), by the widening multiply
    of the top 32 bits (Lemire's method without the rejection step; the bias
    is below 2**-20 for the ranges used here)."""
    w = words(seed, stream, 0, count) >> np.uint64(32)
    span = np.uint64(hi - lo + 1)
    return (lo + ((w * span) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """One NMF problem: V (p x n) ~= W (p x r) @ H (r x n)."""
    name: str
    V: np.ndarray           # float32 (p, n), row-major
    W0: np.ndarray          # float32 (p, r)
    H0: np.ndarray          # float32 (r, n)
    r: int
    iters: int
    eps: float = 1e-10
    seed: int = BASE_SEED

    @property
    def p(self):
        return self.V.shape[0]

    @property
    def n(self):
        return self.V.shape[1]


def starting_factors(seed: int, p: int, n: int, r: int):
    """Algorithm 1's start: W and H iid uniform on (0,1)."""
    return (uniform_open(seed, STREAM_W, (p, r)),
            uniform_open(seed, STREAM_H, (r, n)))


def uniform_problem(p: int, n: int, r: int, seed: int, iters: int = 10,
                    name: str = "uniform", eps: float = 1e-10) -> Problem:
    """V iid uniform on [0,1) (the faces-shaped and tall sweep workloads)."""
    V = uniform_closed_open(seed, STREAM_V, (p, n))
    W0, H0 = starting_factors(seed, p, n, r)
    return Problem(name, V, W0, H0, r, iters, eps, seed)


def exponential_problem(p: int, n: int, r: int, seed: int, iters: int = 20,
                        name: str = "exponential", eps: float = 1e-10) -> Problem:
    """V iid Exponential(1) (the large streaming workload)."""
    V = exponential(seed, STREAM_V, (p, n))
    W0, H0 = starting_factors(seed, p, n, r)
    return Problem(name, V, W0, H0, r, iters, eps, seed)


def planted_problem(p: int, n: int, r: int, seed: int, sigma: float = 0.01,
                    iters: int = 200, name: str = "planted",
                    eps: float = 1e-10) -> Problem:
    """V = W* H* + |N(0, sigma^2)| with W*, H* iid Gamma(1,1).

    The planted product is formed in float64 and rounded once to float32
    together with the noise."""
    Ws = exponential(seed, STREAM_WSTAR, (p, r)).astype(np.float64)
    Hs = exponential(seed, STREAM_HSTAR, (r, n)).astype(np.float64)
    E = abs_normal(seed, STREAM_NOISE, (p, n), sigma).astype(np.float64)
    V = (Ws @ Hs + E).astype(np.float32)
    W0, H0 = starting_factors(seed, p, n, r)
    return Problem(name, V, W0, H0, r, iters, eps, seed)


def poisson_counts(seed: int, stream: int, lam: np.ndarray) -> np.ndarray:
    """Counts v_ij ~ Poisson(lam_ij), float32.  Drawn with numpy's Generator
    seeded by (seed, stream): reproducible within one numpy version (the
    tests draw the inputs once per process for both sides)."""
    rng = np.random.default_rng([int(seed), int(stream)])
    return rng.poisson(lam).astype(np.float32)


def counts_problem(p: int, n: int, r: int, seed: int, mean: float = 5.0,
                   iters: int = 20, name: str = "counts",
                   eps: float = 1e-10) -> Problem:
    """The Poisson model's workload: counts v_ij ~ Poisson(lam_ij) with
    lam = W* H* scaled to mean ``mean`` (W*, H* iid Gamma(1,1)); Algorithm 1's
    uniform(0,1) start."""
    Ws = exponential(seed, STREAM_WSTAR, (p, r)).astype(np.float64)
    Hs = exponential(seed, STREAM_HSTAR, (r, n)).astype(np.float64)
    lam = (Ws @ Hs) * (mean / r)
    V = poisson_counts(seed, STREAM_COUNTS, lam)
    W0, H0 = starting_factors(seed, p, n, r)
    return Problem(name, V, W0, H0, r, iters, eps, seed)


def exact_planted(p: int, n: int, r: int, seed: int) -> Problem:
    """V = W0 H0 exactly representable: W0 and H0 hold small integers on a
    power-of-two grid so that every product and partial sum is exact in
    float32; the starting factors *are* the planted factors (a fixed point
    of the multiplicative updates when eps = 0)."""
    w = words(seed, STREAM_WSTAR, 0, p * r)
    h = words(seed, STREAM_HSTAR, 0, r * n)
    W0 = ((w >> np.uint64(61)).astype(np.float32) + 1.0).reshape(p, r) / 8.0
    H0 = ((h >> np.uint64(61)).astype(np.float32) + 1.0).reshape(r, n) / 4.0
    V = (W0.astype(np.float64) @ H0.astype(np.float64)).astype(np.float32)
    return Problem("exact_planted", V, W0.astype(np.float32), H0.astype(np.float32),
                   r, 10, 0.0, seed)


# The five measured configurations, by what they are.
FACES = dict(name="faces_361x2429_r10", p=361, n=2429, r=10, iters=50)
PLANTED = dict(name="planted_8192x8192_r50", p=8192, n=8192, r=50, iters=200)
TALL = dict(name="tall_65536x4096", p=65536, n=4096, iters=20)
LARGE = dict(name="large_131072x16384_r64", p=131072, n=16384, r=64, iters=20)
BATCH = dict(name="batched_512", count=512, pmin=64, pmax=2048, rmin=4, rmax=32,
             iters=100)
COUNTS = dict(name="counts_8192x8192_r50", p=8192, n=8192, r=50, iters=20)


def tall(r: int, seed: int = BASE_SEED + 2, iters: int = 20) -> Problem:
    c = TALL
    return uniform_problem(c["p"], c["n"], r, seed, iters, f"{c['name']}_r{r}")


def large(seed: int = BASE_SEED + 4, iters: int = 20) -> Problem:
    c = LARGE
    return exponential_problem(c["p"], c["n"], c["r"], seed, iters, c["name"])


def faces(seed: int = BASE_SEED + 0) -> Problem:
    c = FACES
    return uniform_problem(c["p"], c["n"], c["r"], seed, c["iters"], c["name"])


def planted(seed: int = BASE_SEED + 1, p: int = 8192, n: int = 8192,
            r: int = 50, iters: int = 200) -> Problem:
    return planted_problem(p, n, r, seed, 0.01, iters,
                           f"planted_{p}x{n}_r{r}")


def batch_shapes(count: int = 512, seed: int = BASE_SEED + 3,
                 pmin: int = 64, pmax: int = 2048, rmin: int = 4, rmax: int = 32):
    """Per-instance (p, n, r) of the batched workload: p, n iid uniform on
    {pmin..pmax}, r iid uniform on {rmin..rmax}."""
    ps = uniform_int(seed, STREAM_SHAPES, count, pmin, pmax)
    ns = uniform_int(seed + 1, STREAM_SHAPES, count, pmin, pmax)
    rs = uniform_int(seed + 2, STREAM_SHAPES, count, rmin, rmax)
    return [(int(a), int(b), int(c)) for a, b, c in zip(ps, ns, rs)]


def batch(count: int = 512, seed: int = BASE_SEED + 3, iters: int = 100,
          pmin: int = 64, pmax: int = 2048, rmin: int = 4, rmax: int = 32):
    """The batched workload: independent problems with V iid uniform on [0,1);
    instance ``b`` uses seed ``seed * 1000 + b``."""
    probs = []
    for b, (p, n, r) in enumerate(batch_shapes(count, seed, pmin, pmax, rmin, rmax)):
        probs.append(uniform_problem(p, n, r, seed * 1000 + b, iters,
                                     f"batch{b}_{p}x{n}_r{r}"))
    return probs


def counts(seed: int = BASE_SEED + 5, iters: int = 20) -> Problem:
    c = COUNTS
    return counts_problem(c["p"], c["n"], c["r"], seed, 5.0, iters, c["name"])


# ----------------------------------------------------------------------------
# PET reconstruction inputs (Section 3.2): detector geometry, phantom, counts
# ----------------------------------------------------------------------------
#
# A G x G grid of unit pixels fills the square [0, G]^2 (pixel j = row * G +
# col covers [col, col+1] x [row, row+1]); `ndet` detectors sit evenly on a
# circle around it (angles 2 pi (a + 1/2) / ndet, radius a little beyond the
# grid's half diagonal), and every unordered pair of detectors is one line of
# flight, so d = ndet (ndet - 1) / 2 (64 detectors give the 2016 lines of the
# paper's 64 x 64 example).  The geometry constant e_ij is the length of line
# i inside pixel j, computed exactly from the line's crossings of the grid
# lines (Siddon, Med. Phys. 12, 1985).  This is the stand-in for the
# simulated scanner of the paper's example; the method's own first step, the
# scaling of E to unit column sums, is not done here.

def pet_system_matrix(grid: int, ndet: int) -> np.ndarray:
    """E (d x p, float32, row-major): intersection lengths of the ndet
    (ndet - 1) / 2 detector-pair lines with the grid x grid unit pixels."""
    G = int(grid)
    c = G / 2.0
    R = 0.5 * math.sqrt(2.0) * G + 1.0
    ang = 2.0 * math.pi * (np.arange(ndet) + 0.5) / ndet
    det = np.stack([c + R * np.cos(ang), c + R * np.sin(ang)], axis=1)
    ia, ib = np.triu_indices(ndet, 1)
    P0, D = det[ia], det[ib] - det[ia]
    length = np.hypot(D[:, 0], D[:, 1])
    planes = np.arange(G + 1, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        tx = (planes[None, :] - P0[:, :1]) / D[:, :1]
        ty = (planes[None, :] - P0[:, 1:]) / D[:, 1:]
    tx[~np.isfinite(tx)] = np.nan
    ty[~np.isfinite(ty)] = np.nan
    # the part of each line inside the box [0, G]^2
    lo = np.fmax(np.fmin(tx[:, 0], tx[:, -1]), np.fmin(ty[:, 0], ty[:, -1]))
    hi = np.fmin(np.fmax(tx[:, 0], tx[:, -1]), np.fmax(ty[:, 0], ty[:, -1]))
    lo = np.nan_to_num(np.fmax(lo, 0.0), nan=0.0)
    hi = np.nan_to_num(np.fmin(hi, 1.0), nan=0.0)
    t = np.concatenate([tx, ty, lo[:, None], hi[:, None]], axis=1)
    t = np.where((t >= lo[:, None]) & (t <= hi[:, None]), t, np.nan)
    t.sort(axis=1)                                  # NaNs sort last
    dt = t[:, 1:] - t[:, :-1]
    mid = 0.5 * (t[:, 1:] + t[:, :-1])
    x = P0[:, :1] + mid * D[:, :1]
    y = P0[:, 1:] + mid * D[:, 1:]
    ok = np.isfinite(dt) & (dt > 0)
    col = np.floor(np.where(ok, x, -1)).astype(np.int64)
    row = np.floor(np.where(ok, y, -1)).astype(np.int64)
    ok &= (col >= 0) & (col < G) & (row >= 0) & (row < G)
    d = len(ia)
    E = np.zeros((d, G * G), dtype=np.float64)
    li = np.broadcast_to(np.arange(d)[:, None], ok.shape)[ok]
    np.add.at(E, (li, (row * G + col)[ok]), (dt * length[:, None])[ok])
    return E.astype(np.float32)


def pet_phantom(grid: int) -> np.ndarray:
    """True intensities (p, float64) of a synthetic emission image: a
    background disk with brighter and darker elliptical inserts, on the
    grid's pixel centres (relative units; pet_problem scales them)."""
    G = int(grid)
    u = (np.arange(G) + 0.5) / G * 2.0 - 1.0             # pixel centres in [-1, 1]
    X, Y = np.meshgrid(u, u)                              # X: column, Y: row
    img = np.zeros((G, G))
    # (centre x, centre y, semi-axis a, semi-axis b, rotation, added intensity)
    for cx, cy, a, b, th, val in [
            (0.0, 0.0, 0.85, 0.80, 0.0, 1.0),
            (-0.30, 0.15, 0.22, 0.35, 0.4, 2.0),
            (0.35, 0.25, 0.18, 0.12, -0.3, 3.0),
            (0.10, -0.45, 0.30, 0.10, 0.0, -0.6),
            (-0.20, -0.20, 0.08, 0.08, 0.0, 4.0),
            (0.45, -0.10, 0.06, 0.15, 0.8, 2.5)]:
        xr = (X - cx) * math.cos(th) + (Y - cy) * math.sin(th)
        yr = -(X - cx) * math.sin(th) + (Y - cy) * math.cos(th)
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += val
    return img.reshape(-1)


def grid_neighbours(grid: int):
    """The neighbourhood system N of the penalty (Section 3.2): first-order
    (horizontal and vertical) adjacency on the grid, as CSR arrays
    (ptr: p + 1 int32, idx: int32), each pixel's neighbours in the order up,
    left, right, down.  Symmetric: k in N_j exactly when j in N_k."""
    G = int(grid)
    ptr, idx = [0], []
    for r in range(G):
        for c in range(G):
            for rr, cc in ((r - 1, c), (r, c - 1), (r, c + 1), (r + 1, c)):
                if 0 <= rr < G and 0 <= cc < G:
                    idx.append(rr * G + cc)
            ptr.append(len(idx))
    return np.asarray(ptr, dtype=np.int32), np.asarray(idx, dtype=np.int32)


@dataclasses.dataclass
class PetProblem:
    """One PET reconstruction: counts y (d) along the lines of E (d x p,
    raw geometry), the neighbourhood CSR and the penalty constants mu (one
    image per value), started from lambda = 1 (Algorithm 2)."""
    name: str
    E: np.ndarray          # float32 (d, p), row-major, unscaled lengths
    y: np.ndarray          # float32 (d,), counts
    nbr_ptr: np.ndarray    # int32 (p + 1,)
    nbr_idx: np.ndarray    # int32 (nnz,)
    mu: tuple
    iters: int
    grid: int
    lam_true: np.ndarray   # float64 (p,), the phantom the counts were drawn from

    @property
    def d(self):
        return self.E.shape[0]

    @property
    def p(self):
        return self.E.shape[1]


def pet_problem(grid: int, ndet: int, seed: int, mean_count: float = 20.0,
                mu=(0.0, 1e-7, 1e-6, 1e-5), iters: int = 10,
                name: str = "pet") -> PetProblem:
    """y_i ~ Poisson((E lam_true)_i) with the phantom scaled so the mean
    expected count per line is `mean_count`; numpy's Generator seeded by
    (seed, STREAM_PET_COUNTS)."""
    E = pet_system_matrix(grid, ndet)
    lam = pet_phantom(grid)
    proj = E.astype(np.float64) @ lam
    lam = lam * (mean_count / proj.mean())
    rng = np.random.default_rng([int(seed), STREAM_PET_COUNTS])
    y = rng.poisson(E.astype(np.float64) @ lam).astype(np.float32)
    ptr, idx = grid_neighbours(grid)
    return PetProblem(name, E, y, ptr, idx, tuple(float(m) for m in mu), iters, grid, lam)


PET = dict(name="pet_64x64_d2016", grid=64, ndet=64, iters=100)
PET_LARGE = dict(name="pet_128x128_d8128", grid=128, ndet=128, iters=20)
# Penalty constants of the workloads: four decades like the paper's table,
# placed for this phantom's intensity scale (unit-column-sum E, about 20
# expected counts per line), where the paper's own values (1e-7 .. 1e-5,
# for its data's scale) would all act like mu = 0.
PET_MU = (0.0, 1e-4, 1e-3, 1e-2)


def pet(seed: int = BASE_SEED + 6, iters: int = None) -> PetProblem:
    """The paper's PET example shape: 64 x 64 pixels, 2016 lines."""
    c = PET
    return pet_problem(c["grid"], c["ndet"], seed, mu=PET_MU, iters=iters or c["iters"],
                       name=c["name"])


def pet_large(seed: int = BASE_SEED + 7, iters: int = None) -> PetProblem:
    """A larger scanner: 128 x 128 pixels, 128 detectors, 8128 lines (E is
    532 MB, four times the L2 cache)."""
    c = PET_LARGE
    return pet_problem(c["grid"], c["ndet"], seed, mu=PET_MU, iters=iters or c["iters"],
                       name=c["name"])
