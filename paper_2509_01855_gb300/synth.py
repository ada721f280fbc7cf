"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle legs.

This module holds none of the method's arithmetic: it draws random vectors, random Chebyshev
mode lists, initial guesses from closed-form physics (evaluated at node times that the caller
supplies) and request streams. Base seed 2509_01855; each stream derives its own seed with
numpy's SeedSequence.
"""
import numpy as np

BASE_SEED = 2509_01855


def rng(*tags):
    """Generator for a named stream: SeedSequence(BASE_SEED, spawn key = tags)."""
    key = tuple(int(t) if isinstance(t, (int, np.integer)) else sum(map(ord, str(t))) for t in tags)
    return np.random.default_rng(np.random.SeedSequence(BASE_SEED, spawn_key=key))


def gaussian(shape, *tags):
    """Standard normal FP64 array."""
    return rng("gauss", *tags).standard_normal(shape)


def sparse_modes(N, n_random=26, *tags):
    """Chebyshev mode list {0, 1, 2, N-2, N-1, N} plus n_random distinct modes in [3, N-3],
    and standard-normal amplitudes."""
    g = rng("modes", N, *tags)
    fixed = [0, 1, 2, N - 2, N - 1, N]
    pool = max(0, N - 5)
    extra = []
    if pool > 0:
        extra = list(3 + g.choice(pool, size=min(n_random, pool), replace=False))
    modes = sorted(set(fixed + [int(m) for m in extra]))
    return modes, g.standard_normal(len(modes))


def orbit_guess(t, rf, tf, t0=0.0):
    """Tangential-thrust spiral from the unit circular orbit that ends at radius r_f at tf:
    v(t) = 1 - a_e (t - t0), a_e = (1 - r_f^-1/2)/(tf - t0); r = 1/v^2, theta = (1 - v^4)/(4 a_e),
    v_r = 2 a_e / v^3, v_theta = v, thrust (0, a_e). Returns X (4, L), U (2, L)."""
    t = np.asarray(t, dtype=np.float64)
    ae = (1.0 - rf ** -0.5) / (tf - t0)
    v = 1.0 - ae * (t - t0)
    X = np.stack([1.0 / v**2, (1.0 - v**4) / (4.0 * ae), 2.0 * ae / v**3, v])
    U = np.zeros((2, t.size))
    U[1] = ae
    return X, U


def double_integrator_guess(t, t0=0.0, tf=1.0):
    """Boundary states (0,0) -> (1,0) joined linearly in time, u = 0."""
    lam = (np.asarray(t, dtype=np.float64) - t0) / (tf - t0)
    X = np.stack([lam, np.zeros_like(lam)])
    return X, np.zeros((1, lam.size))


def smooth_coefficient(t, t0, tf, *tags, n_modes=8, mean=-1.0, amp=0.5):
    """d(t) = mean + amp * sum_k c_k cos(k theta), theta = arccos of t mapped to [-1, 1],
    c_k ~ N(0, 1) / (k + 1), normalised to unit max |c|; the smooth variable coefficient of the
    scalar linear-solve experiment."""
    g = rng("dsmooth", *tags)
    c = g.standard_normal(n_modes) / (np.arange(n_modes) + 1.0)
    c /= np.abs(c).sum()
    x = np.clip(2.0 * (np.asarray(t) - t0) / (tf - t0) - 1.0, -1.0, 1.0)
    th = np.arccos(x)
    return mean + amp * sum(c[k] * np.cos(k * th) for k in range(n_modes))


def rough_coefficient(L, *tags, mean=-1.0, amp=0.5):
    """d_i = mean + amp * N(0, 1) per node (rough variant)."""
    return mean + amp * rng("drough", *tags).standard_normal(L)


def serving_requests(n, rate, *tags, kmin=8, kmax=16, rf_range=(1.2, 2.0), tf_range=(10.0, 30.0)):
    """Poisson arrivals (exponential gaps of mean 1/rate) with N = 2^k, k ~ U{kmin..kmax},
    r_f ~ U(rf_range), t_f ~ U(tf_range). Returns a list of dicts sorted by arrival time."""
    g = rng("serve", *tags)
    gaps = g.exponential(1.0 / rate, n)
    arr = np.cumsum(gaps)
    ks = g.integers(kmin, kmax + 1, n)
    rfs = g.uniform(*rf_range, n)
    tfs = g.uniform(*tf_range, n)
    return [dict(id=i, arrival=float(arr[i]), N=int(1 << ks[i]), rf=float(rfs[i]),
                 tf=float(tfs[i])) for i in range(n)]
