"""Seeded synthetic workloads for the regular-force step.

This module is shared by the CUDA path's tests/benchmarks and by the oracle's
tests.  It holds only the *models* the paper's experiments are built from
(Plummer and King W0=6 star clusters, the Kroupa 2001 mass function, primordial
binaries entering as centre-of-mass particles, a power-of-two block-step
histogram and a neighbour radius) and none of the method's arithmetic: no
pairwise force, jerk, potential, prediction or neighbour test lives here.

Units are N-body (Henon) units, G = M = 1, E = -1/4 (Sec. 3.3.2 of the paper
names the units; Heggie & Mathieu 1986 define them).

Every generator takes an integer seed and uses numpy's PCG64 stream, so the same
seed gives the same bits on any host.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PLUMMER_A_NBODY = 3.0 * math.pi / 16.0  # Plummer scale length giving E = -1/4 (G = M = 1)
PC_PER_AU = 1.0 / 206264.806


# --------------------------------------------------------------------------
# Mass functions
# --------------------------------------------------------------------------
KROUPA_BREAKS = (0.08, 0.5, 100.0)   # Msun; Kroupa (2001) two-segment IMF as used in Sec. 4.1
KROUPA_SLOPES = (1.3, 2.3)           # dN/dm ∝ m^-alpha on each segment, continuous at 0.5


def _powerlaw_integral(lo, hi, p):
    """∫_lo^hi m^p dm."""
    if abs(p + 1.0) < 1e-15:
        return math.log(hi / lo)
    return (hi ** (p + 1.0) - lo ** (p + 1.0)) / (p + 1.0)


def kroupa_segment_weights(breaks=KROUPA_BREAKS, slopes=KROUPA_SLOPES):
    """Relative number in each IMF segment (continuous at the break)."""
    (m0, m1, m2), (a1, a2) = breaks, slopes
    # xi(m) = m^-a1 on [m0,m1); xi(m) = m1^(a2-a1) m^-a2 on [m1,m2]
    c2 = m1 ** (a2 - a1)
    w1 = _powerlaw_integral(m0, m1, -a1)
    w2 = c2 * _powerlaw_integral(m1, m2, -a2)
    return np.array([w1, w2]) / (w1 + w2)


def kroupa_masses(n: int, rng: np.random.Generator, breaks=KROUPA_BREAKS,
                  slopes=KROUPA_SLOPES) -> np.ndarray:
    """Draw n masses (Msun) from the two-segment Kroupa (2001) IMF by inverse CDF."""
    w = kroupa_segment_weights(breaks, slopes)
    seg = (rng.random(n) >= w[0]).astype(np.int64)
    u = rng.random(n)
    out = np.empty(n)
    for s in (0, 1):
        lo, hi, a = breaks[s], breaks[s + 1], slopes[s]
        p = 1.0 - a
        sel = seg == s
        out[sel] = (lo ** p + u[sel] * (hi ** p - lo ** p)) ** (1.0 / p)
    return out


# --------------------------------------------------------------------------
# Plummer sphere
# --------------------------------------------------------------------------
def _isotropic(rng, n):
    cth = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def plummer_positions_velocities(n: int, rng: np.random.Generator, a: float = PLUMMER_A_NBODY,
                                 x_max: float = 0.999):
    """Sample the Plummer distribution function (total mass 1, G = 1).

    Radii by inverting the cumulative mass M(r) = r^3 / (r^2 + a^2)^(3/2) on
    X ~ U(0, x_max) (the truncation keeps r finite); speeds q * v_esc(r) with q
    drawn by rejection from g(q) = q^2 (1 - q^2)^(7/2) (the isotropic Plummer DF).
    """
    X = rng.random(n) * x_max
    X = np.where(X <= 0.0, 1e-300, X)
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(rng, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.random(todo.size)
        yy = 0.1 * rng.random(todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    v_esc = math.sqrt(2.0) * (1.0 + r * r / (a * a)) ** (-0.25) / math.sqrt(a)
    vel = (q * v_esc)[:, None] * _isotropic(rng, n)
    return pos, vel


def plummer_enclosed_mass(r, a: float = PLUMMER_A_NBODY):
    r = np.asarray(r, dtype=np.float64)
    return r ** 3 / (r * r + a * a) ** 1.5


def plummer_potential_energy(a: float = PLUMMER_A_NBODY) -> float:
    """Self potential energy of an (untruncated) Plummer sphere, G = M = 1: -3π/(32 a)."""
    return -3.0 * math.pi / (32.0 * a)


def _to_com_frame(m, x, v):
    mt = m.sum()
    x = x - (m[:, None] * x).sum(0) / mt
    v = v - (m[:, None] * v).sum(0) / mt
    return x, v


# --------------------------------------------------------------------------
# King (1966) model
# --------------------------------------------------------------------------
def _king_rho(W):
    from scipy.special import erf
    W = np.maximum(W, 0.0)
    return np.exp(W) * erf(np.sqrt(W)) - np.sqrt(4.0 * W / math.pi) * (1.0 + 2.0 * W / 3.0)


@dataclass
class KingModel:
    W0: float
    r: np.ndarray            # radius grid, King radius r0 = 1
    W: np.ndarray            # dimensionless potential W(r), W(r_t) = 0
    M: np.ndarray            # enclosed mass, normalised to 1 at r_t
    r_t: float
    concentration: float     # log10(r_t / r0)
    potential_energy: float  # -∫ M dM / r   (G = 1, M_tot = 1, r0 = 1)
    mean_v2: float           # mass-weighted <v^2> in units of sigma^2
    v_scale_to_r0: float = field(default=1.0)


def king_model(W0: float = 6.0, n_grid: int = 4000) -> KingModel:
    """Solve King's Poisson equation for the lowered isothermal sphere.

    In King units (r0 = 1, sigma = 1): W'' + 2 W'/r = -9 rho(W)/rho(W0),
    W(0) = W0, W'(0) = 0, integrated outwards until W = 0 (the tidal radius).
    """
    from scipy.integrate import solve_ivp, cumulative_trapezoid
    rho0 = _king_rho(np.array(W0))

    def rhs(r, y):
        Wr, dW, _ = y
        rr = max(r, 1e-12)
        rho = _king_rho(np.array(Wr)) / rho0
        return [dW, -9.0 * rho - 2.0 * dW / rr, 4.0 * math.pi * rr * rr * rho]

    def hit_zero(r, y):
        return y[0]
    hit_zero.terminal = True
    hit_zero.direction = -1
    r_start = 1e-6
    sol = solve_ivp(rhs, [r_start, 1e4], [W0, -3.0 * r_start, 0.0], events=hit_zero,
                    rtol=1e-11, atol=1e-13, dense_output=True)
    r_t = float(sol.t_events[0][0])
    r = np.concatenate([[0.0], np.geomspace(1e-4, r_t, n_grid)])
    y = sol.sol(np.maximum(r, r_start))
    W = np.clip(y[0], 0.0, None)
    W[0] = W0
    Mraw = np.where(r > 0, y[2], 0.0)
    Mtot = Mraw[-1]
    M = Mraw / Mtot
    dM = np.gradient(M, r)
    integrand = np.where(r > 0, M * dM / np.maximum(r, 1e-300), 0.0)
    pot_energy = -float(cumulative_trapezoid(integrand, r)[-1])
    # In King units G*rho0 = 9/(4π); with M_tot as computed the potential energy
    # in (G=1, M=1, r0=1) units is pot_energy; velocities are measured in sigma.
    # <v^2>(W) for f ∝ e^{W - v^2/2} - 1 on v < sqrt(2W):
    vg = np.linspace(0.0, 1.0, 401)

    def moments(Wv):
        if Wv <= 0:
            return 0.0, 0.0
        vmax = math.sqrt(2.0 * Wv)
        v = vg * vmax
        f = np.exp(Wv - 0.5 * v * v) - 1.0
        m2 = np.trapezoid(v * v * f, v)
        m4 = np.trapezoid(v ** 4 * f, v)
        return m2, m4
    mv = np.array([moments(w) for w in W])
    v2 = np.where(mv[:, 0] > 0, mv[:, 1] / np.maximum(mv[:, 0], 1e-300), 0.0)
    mean_v2 = float(np.trapezoid(v2 * dM, r))
    return KingModel(W0=W0, r=r, W=W, M=M, r_t=r_t, concentration=math.log10(r_t),
                     potential_energy=pot_energy, mean_v2=mean_v2)


def king_positions_velocities(n: int, rng: np.random.Generator, model: KingModel):
    """Sample positions and velocities (King units: r0 = 1, sigma = 1)."""
    u = rng.random(n)
    r = np.interp(u, model.M, model.r)
    W = np.interp(r, model.r, model.W)
    pos = r[:, None] * _isotropic(rng, n)
    speed = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        Wt = W[todo]
        vmax = np.sqrt(2.0 * np.maximum(Wt, 0.0))
        v = vmax * rng.random(todo.size)
        # p(v) ∝ v^2 (e^{W - v^2/2} - 1), bounded by vmax^2 (e^W - 1)
        fmax = vmax * vmax * np.expm1(Wt)
        y = fmax * rng.random(todo.size)
        ok = (y < v * v * np.expm1(Wt - 0.5 * v * v)) | (vmax == 0.0)
        speed[todo[ok]] = np.where(vmax[ok] == 0.0, 0.0, v[ok])
        todo = todo[~ok]
    vel = speed[:, None] * _isotropic(rng, n)
    return pos, vel, r


# --------------------------------------------------------------------------
# Cluster containers
# --------------------------------------------------------------------------
@dataclass
class Cluster:
    """A particle set in N-body units.  Arrays are float64; x, v are (n, 3)."""
    m: np.ndarray
    x: np.ndarray
    v: np.ndarray
    model: str
    seed: int
    enclosed_mass: object = None      # callable r -> M(<r) of the parent model (N-body units)
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.m.shape[0]


def plummer(n: int, seed: int, masses: str = "equal", x_max: float = 0.999,
            com: bool = True) -> Cluster:
    """Plummer sphere in N-body units (a = 3π/16), equal or Kroupa masses (Σm = 1)."""
    rng = np.random.default_rng(seed)
    if masses == "equal":
        m = np.full(n, 1.0 / n)
    elif masses == "kroupa":
        m = kroupa_masses(n, rng)
        m = m / m.sum()
    else:
        raise ValueError(masses)
    x, v = plummer_positions_velocities(n, rng, x_max=x_max)
    if com:
        x, v = _to_com_frame(m, x, v)
    return Cluster(m=m, x=np.ascontiguousarray(x), v=np.ascontiguousarray(v), model="plummer",
                   seed=seed, enclosed_mass=plummer_enclosed_mass)


def king(n: int, seed: int, W0: float = 6.0, masses: str = "kroupa",
         binary_fraction: float = 0.0, R_h_pc: float = 7.5) -> Cluster:
    """King (1966) W0 model in N-body units, Kroupa masses, optional binary c.m. particles.

    A fraction `binary_fraction` of the n particle slots becomes the centre of mass
    of a primordial binary: its mass is m1 + m2 (two IMF draws), it sits at the
    sampled position/velocity, and the binary's semi-major axis (log-uniform in
    0.005 - 50 AU, converted with the 7.5 pc half-mass radius of the paper's
    million-body model, Sec. 5) is recorded but does not enter the regular force.
    """
    rng = np.random.default_rng(seed)
    model = king_model(W0)
    m = kroupa_masses(n, rng)
    nb = int(round(binary_fraction * n))
    bin_idx = np.sort(rng.choice(n, size=nb, replace=False)) if nb else np.zeros(0, np.int64)
    if nb:
        m2 = kroupa_masses(nb, rng)
        m[bin_idx] += m2
    m = m / m.sum()
    x, v, _ = king_positions_velocities(n, rng, model)
    # Scale to N-body units using the model's own energies (virial equilibrium):
    # lengths so that W = -1/2, speeds so that <v^2> = 1/2.
    lam = -2.0 * model.potential_energy
    x = x * lam
    v = v * math.sqrt(0.5 / model.mean_v2)
    x, v = _to_com_frame(m, x, v)
    rr, MM = model.r * lam, model.M

    def enclosed(r):
        return np.interp(np.asarray(r, dtype=np.float64), rr, MM)
    extra = {"W0": W0, "r_t": model.r_t * lam, "concentration": model.concentration}
    if nb:
        lg = rng.uniform(math.log(0.005), math.log(50.0), nb)
        a_au = np.exp(lg)
        rh_model = float(np.interp(0.5, MM, rr))
        extra.update(binary_index=bin_idx, binary_a_au=a_au,
                     binary_a_nbody=a_au * PC_PER_AU * rh_model / R_h_pc)
    return Cluster(m=m, x=np.ascontiguousarray(x), v=np.ascontiguousarray(v), model="king",
                   seed=seed, enclosed_mass=enclosed, extra=extra)


# --------------------------------------------------------------------------
# Workload parameters: neighbour radius and active blocks
# --------------------------------------------------------------------------
def neighbour_radius2(x: np.ndarray, target: int, seed: int = 0, sample: int = 16384) -> float:
    """Global r_s^2 for which the median neighbour count is about `target`.

    Uses a k-d tree (scipy) k-nearest-neighbour query on a seeded sample of
    particles: r_s is the median distance to the target-th nearest other particle,
    nudged up by 1e-9 so that a particle at exactly that distance counts.
    """
    from scipy.spatial import cKDTree
    n = x.shape[0]
    if target >= n:
        raise ValueError("target neighbour count must be < n")
    rng = np.random.default_rng(seed)
    q = x if n <= sample else x[rng.choice(n, size=sample, replace=False)]
    tree = cKDTree(x)
    d, _ = tree.query(q, k=target + 1)
    rs = float(np.median(d[:, target])) * (1.0 + 1e-9)
    return rs * rs


def block_steps(cluster: Cluster, eta: float = 0.05, scatter: float = 0.5, seed: int = 0,
                dt_min: float = 0.5 ** 22, dt_max: float = 0.5 ** 3) -> np.ndarray:
    """Power-of-two block steps from the parent model's local dynamical time.

    dt_i = 2^floor(log2(eta * t_dyn(r_i) * s_i)) with t_dyn = sqrt(r^3 / M(<r)) of
    the parent model (G = 1) and s_i a seeded log-normal scatter, clipped to
    [2^-22, 2^-3] (Sec. 3.3.1: steps are integer powers of 0.5, the deepest
    levels reach 0.5^20 - 0.5^22).  Particles in the dense core get the
    smallest steps, as in a block-step run.
    """
    rng = np.random.default_rng(seed + 7919)
    r = np.sqrt((cluster.x ** 2).sum(1))
    M = np.maximum(cluster.enclosed_mass(r), 1e-300)
    tdyn = np.sqrt(np.maximum(r, 1e-12) ** 3 / M)
    s = np.exp(scatter * rng.standard_normal(r.shape[0]))
    dt = 2.0 ** np.floor(np.log2(eta * tdyn * s))
    return np.clip(dt, dt_min, dt_max)


def sorted_step_list(steps: np.ndarray) -> np.ndarray:
    """Particle indices sorted by (step, index): the time-step sorting list of Sec. 3.3.1."""
    return np.lexsort((np.arange(steps.shape[0]), steps)).astype(np.int64)


def active_block(steps: np.ndarray, n_i: int) -> np.ndarray:
    """The first n_i entries of the sorting list (int32): the particles with the smallest steps."""
    order = sorted_step_list(steps)
    return np.ascontiguousarray(order[:n_i].astype(np.int32))


# --------------------------------------------------------------------------
# Predictor inputs (Hermite state at the last step) — synthetic
# --------------------------------------------------------------------------
def hermite_state(cluster: Cluster, seed: int, t_block: float = 0.0, steps: np.ndarray | None = None,
                  acc_scale: float = 1.0, jerk_scale: float = 10.0):
    """Synthetic (a, jerk, t_last) for a predictor call.

    The predictor only needs some force and jerk at each particle's last step
    time; here they are seeded Gaussian vectors of N-body-unit magnitude, and
    t_last_i = t_block - k_i * dt_i with k_i in {0, 1} so that t_block - t_last
    spans zero and one block step.
    """
    rng = np.random.default_rng(seed + 104729)
    n = cluster.n
    a = acc_scale * rng.standard_normal((n, 3))
    j = jerk_scale * rng.standard_normal((n, 3))
    if steps is None:
        steps = np.full(n, 0.5 ** 6)
    k = rng.integers(0, 2, n)
    t_last = t_block - k * steps
    return np.ascontiguousarray(a), np.ascontiguousarray(j), np.ascontiguousarray(t_last)


# --------------------------------------------------------------------------
# Ensemble of independent clusters
# --------------------------------------------------------------------------
@dataclass
class Ensemble:
    m: np.ndarray
    x: np.ndarray
    v: np.ndarray
    cluster_off: np.ndarray   # int64 [C+1] particle offsets
    active_off: np.ndarray    # int64 [C+1] offsets into idx
    idx: np.ndarray           # int32 global active indices (cluster-major)
    rs2: np.ndarray           # float64 [C] per-cluster r_s^2
    sizes: np.ndarray
    fractions: np.ndarray


def ensemble(n_clusters: int = 512, seed: int = 4, n_lo: int = 256, n_hi: int = 32768,
             nb_target: int = 50, frac_lo: float = 1.0 / 64.0, frac_hi: float = 1.0) -> Ensemble:
    """Independent equal-mass Plummer clusters with log-uniform N and uniform active fractions."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_clusters))).astype(np.int64)
    fracs = rng.uniform(frac_lo, frac_hi, n_clusters)
    ms, xs, vs, idxs, rs2 = [], [], [], [], []
    off = np.zeros(n_clusters + 1, np.int64)
    aoff = np.zeros(n_clusters + 1, np.int64)
    for c in range(n_clusters):
        cl = plummer(int(sizes[c]), seed=seed * 100003 + c)
        steps = block_steps(cl, seed=seed * 100003 + c)
        ni = max(1, int(math.ceil(fracs[c] * cl.n)))
        act = active_block(steps, ni).astype(np.int64) + off[c]
        ms.append(cl.m); xs.append(cl.x); vs.append(cl.v); idxs.append(act)
        rs2.append(neighbour_radius2(cl.x, min(nb_target, cl.n - 1), seed=c, sample=2048))
        off[c + 1] = off[c] + cl.n
        aoff[c + 1] = aoff[c] + ni
    return Ensemble(m=np.concatenate(ms), x=np.ascontiguousarray(np.concatenate(xs)),
                    v=np.ascontiguousarray(np.concatenate(vs)), cluster_off=off, active_off=aoff,
                    idx=np.concatenate(idxs).astype(np.int32), rs2=np.array(rs2), sizes=sizes,
                    fractions=fracs)


# --------------------------------------------------------------------------
# The named workloads
# --------------------------------------------------------------------------
def plummer_1k_equal(seed: int = 0):
    """Plummer N = 1024, equal masses, r_s for a median of ~50 neighbours."""
    cl = plummer(1024, seed)
    return cl, neighbour_radius2(cl.x, 50, seed=seed)


def plummer_128k_kroupa(seed: int = 1):
    """Plummer N = 131072 with Kroupa masses, r_s for a median of ~80 neighbours (cap 512)."""
    cl = plummer(131072, seed, masses="kroupa")
    return cl, neighbour_radius2(cl.x, 80, seed=seed)


def king_1m_binaries(seed: int = 2, n: int = 1 << 20):
    """King W0 = 6, N = 2^20 j-particles incl. 5% binary c.m. particles, Kroupa masses."""
    cl = king(n, seed, W0=6.0, masses="kroupa", binary_fraction=0.05)
    return cl, neighbour_radius2(cl.x, 80, seed=seed)


def plummer_64k_kroupa(seed: int = 3):
    cl = plummer(65536, seed, masses="kroupa")
    return cl, neighbour_radius2(cl.x, 80, seed=seed)


# --------------------------------------------------------------------------
# Step levels for the block-step scheduler
# --------------------------------------------------------------------------
def step_levels(steps: np.ndarray) -> np.ndarray:
    """Level k of each power-of-two step 2^-k (int32)."""
    k = np.rint(-np.log2(steps)).astype(np.int32)
    if not np.all(np.ldexp(1.0, -k) == steps):
        raise ValueError("steps must be integer powers of two")
    return k


def level_requests(levels: np.ndarray, seed: int, p_double: float = 0.2, p_halve: float = 0.15,
                   p_halve2: float = 0.05) -> np.ndarray:
    """Seeded requested next levels for the particles of one block step: a stand-in for the
    step criterion of the integrator, which asks for a larger step (level - 1), a smaller one
    (level + 1 or + 2) or the same.  Whether a request is granted is the scheduler's rule."""
    rng = np.random.default_rng(seed)
    u = rng.random(levels.shape[0])
    d = np.zeros(levels.shape[0], np.int32)
    d[u < p_double] = -1
    d[(u >= p_double) & (u < p_double + p_halve)] = 1
    d[(u >= p_double + p_halve) & (u < p_double + p_halve + p_halve2)] = 2
    return (levels + d).astype(np.int32)
