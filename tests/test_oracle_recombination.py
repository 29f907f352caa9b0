"""Pins of the oracle's recombination reactions (Sec. 5.1, the air chemistry
table: e + M+ -> 0 with propensity k_ep X_e X_+, M- + M+ -> 0 with k_np X_+
X_-, k = beta / dV) inside the per-cell hybrid tau-leap/SSA (Sec. 3.2.3).

Three kinds of independent reference:

* below the critical threshold every reaction runs as SSA, which samples
  the chemical master equation exactly: the distribution of the final counts
  over many independent cells is compared with the master equation's
  solution, exp(Q t) of the finite generator built here from the table's
  propensities (scipy's matrix exponential);
* far above it the tau-leap of Cao et al. (2006) with the bound eps and
  g = 2 (a second-order reaction of distinct reactants) takes, in the mean,
  X -> X (1 - eps/2) per leap for X_e = X_+ = X; the exact solution of
  dX/dt = -k X^2 is 1/X = 1/X0 + k t, and summing the local error -eps^2/4
  damped by (X_f/X_n)^2 gives the mean relative bias -(eps/2)(1 - X_f/X0)
  to first order in eps -- so a wrong g, a dropped reactant or a halved
  propensity moves the mean by a multiple of the tolerance;
* whole steps: the net charge sum(N+) - sum(N-) - sum(w) changes only by the
  electrons absorbed at the walls, every count stays non-negative.
"""
import numpy as np
import pytest
from scipy import linalg, stats

from paper_2307_01797_gb300 import synth

NU = np.array([[+1, +1, 0], [-1, 0, +1], [0, 0, 0], [-1, -1, 0], [0, -1, -1]], np.int64)


def _props(kr, X):
    xe, xp, xm = (float(v) for v in X)
    return np.array([kr[0] * xe, kr[1] * xe, kr[2] * xe, kr[3] * xe * xp, kr[4] * xp * xm])


def _master_equation(X0, kr, t):
    """Distribution at time t of the counts (X_e, X_+, X_-) from X0 under the
    table's propensities; ionization off (a finite state space)."""
    assert kr[0] == 0.0
    X0 = tuple(int(v) for v in X0)
    index, states, todo = {X0: 0}, [X0], [X0]
    while todo:
        X = todo.pop()
        for r in range(5):
            if kr[r] <= 0.0 or not NU[r].any():
                continue
            Y = tuple(int(v) for v in np.asarray(X) + NU[r])
            if min(Y) >= 0 and Y not in index:
                index[Y] = len(states)
                states.append(Y)
                todo.append(Y)
    m = len(states)
    Q = np.zeros((m, m))
    for i, X in enumerate(states):
        a = _props(kr, X)
        for r in range(5):
            if a[r] <= 0.0 or not NU[r].any():
                continue
            j = index[tuple(int(v) for v in np.asarray(X) + NU[r])]
            Q[i, j] += a[r]
            Q[i, i] -= a[r]
    P = linalg.expm(Q * t)[0]
    return states, P


def _chi2_against(samples, states, P, alpha=1e-4):
    """Pearson's statistic of the sampled counts against P, bins with fewer
    than 5 expected pooled; returns (statistic, critical value)."""
    index = {s: i for i, s in enumerate(states)}
    obs = np.zeros(len(states))
    for s in samples:
        obs[index[tuple(int(v) for v in s)]] += 1
    n = len(samples)
    exp = P * n
    big = exp >= 5
    o = np.append(obs[big], obs[~big].sum())
    e = np.append(exp[big], exp[~big].sum())
    keep = e > 0
    o, e = o[keep], e[keep]
    stat = float(((o - e) ** 2 / e).sum())
    return stat, float(stats.chi2.ppf(1 - alpha, len(e) - 1))


def _kr(k_ion=0.0, k_att=0.0, k_ph=0.0, k_ep=0.0, k_np=0.0):
    return [k_ion, k_att, k_ph, k_ep, k_np]


@pytest.mark.parametrize("X0,rates", [
    ((4, 6, 0), dict(k_ep=0.05)),                                 # e-ion only
    ((0, 3, 7), dict(k_np=0.05)),                                 # ion-ion only
    ((3, 6, 2), dict(k_att=0.3, k_ph=0.2, k_ep=0.04, k_np=0.06)),  # all but ionization
])
def test_ssa_regime_samples_the_master_equation(oracle_mod, X0, rates):
    """Counts below the critical threshold N_c = 5: the cell is pure SSA, and
    the final counts of 20000 independent cells follow exp(Q dt).  The
    rates are given as k dt; Q uses the propensities of the table (X_e X_+,
    X_+ X_-), so a propensity on X_+ - 1, a missing ion decrement or a
    reaction chosen from the wrong cumulative sum fails the test."""
    ph = synth.physics_small(16)
    p = oracle_mod.make_params(ph, seed=21)
    kr = np.array(_kr(**rates)) / p.dt
    M = 20000
    out = np.array([oracle_mod.kmc_network(p, X0, kr, i)[0] for i in range(M)])
    states, P = _master_equation(X0, kr, p.dt)
    stat, crit = _chi2_against(out, states, P)
    assert stat < crit, (stat, crit)
    # the sampled state space moved: not a test of the initial state alone
    assert (out != np.asarray(X0)).any(axis=1).mean() > 0.3


def test_ssa_regime_detects_a_wrong_propensity(oracle_mod):
    """The statistic above has the power to tell k X_e X_+ from k X_e
    (X_+ - 1): the same samples against the master equation of the wrong
    propensity exceed the critical value many times over."""
    ph = synth.physics_small(16)
    p = oracle_mod.make_params(ph, seed=21)
    X0, k = (4, 6, 0), 0.05 / p.dt
    out = np.array([oracle_mod.kmc_network(p, X0, _kr(k_ep=k), i)[0] for i in range(20000)])
    # wrong propensity k X_e (X_+ - 1), as a generator on the same states
    states = [(e, 2 + e, 0) for e in range(5)]
    Q = np.zeros((5, 5))
    for e in range(1, 5):
        a = k * e * (2 + e - 1)
        Q[e, e - 1] += a
        Q[e, e] -= a
    P_wrong = linalg.expm(Q * p.dt)[4]
    stat, crit = _chi2_against(out, states, P_wrong)
    assert stat > 5 * crit, (stat, crit)


def _leap_bias(eps, X0, Xf, c):
    """First-order (in eps) relative mean bias of the eps-leap for
    dX/dt = -k X (X + c): each leap X -> X (1 - eps/2) (the electrons'
    bound eps X / (2 k X (X + c)) is the tighter one), local error
    -eps^2 X (2X + c) / (8 (X + c)) against the exact flow, damped to the end
    by X_f (X_f + c) / (X_n (X_n + c)), summed as an integral over the
    geometric X_n:  -(eps/4) (X_f + c) [I(X0) - I(X_f)] with
    I(X) = ln(X / (X + c)) / c - 1 / (X + c); c = 0 gives
    -(eps/2)(1 - X_f/X0)."""
    if c == 0:
        return -(eps / 2) * (1.0 - Xf / X0)
    I = lambda X: np.log(X / (X + c)) / c - 1.0 / (X + c)    # noqa: E731
    return -(eps / 4) * (Xf + c) * (I(X0) - I(Xf))


# (reaction, index of the scarcer reactant, k X0 dt, c / X0): the scarcer
# reactant's bound eps X / 2 is the tighter one, so each case pins the g and
# the reactant flag of that species
LEAP_CASES = [
    ("ep", 0, 0.3, 0.0), ("ep", 0, 1.0, 0.0), ("ep", 0, 3.0, 0.0), ("ep", 0, 1.0, 0.5), ("ep", 0, 3.0, 0.5),
    ("ep", 0, 1.0, 2.0), ("ep", 1, 1.0, 0.5), ("np", 1, 1.0, 0.5), ("np", 2, 1.0, 0.5), ("np", 2, 1.0, 0.0),
]


@pytest.mark.parametrize("eps", [0.03, 0.1])
@pytest.mark.parametrize("reaction,small,kX0dt,cfrac", LEAP_CASES)
def test_tau_leap_mean_follows_the_rate_equation(oracle_mod, eps, reaction, small, kX0dt, cfrac):
    """One recombination on, its scarcer reactant at X0 = 10^6 and the other
    at X0 + c: the mean over 200 cells of the scarcer count against the exact
    solution of dX/dt = -k X (X + c), X(t) = c X0 / ((X0 + c) e^{kct} - X0)
    (1/X = 1/X0 + k t for c = 0), with the leap's predicted first-order
    bias; tolerance four standard errors plus eps^2.  The difference of the
    two reactants stays c exactly (same stoichiometry), the third species
    does not move."""
    ph = dict(synth.physics_small(16), eps=eps)
    p = oracle_mod.make_params(ph, seed=5)
    X0 = 10 ** 6
    c = int(cfrac * X0)
    k = kX0dt / (X0 * p.dt)
    pair = (0, 1) if reaction == "ep" else (1, 2)
    other = pair[1] if small == pair[0] else pair[0]
    start = [0, 0, 0]
    start[small], start[other] = X0, X0 + c
    kr = _kr(k_ep=k) if reaction == "ep" else _kr(k_np=k)
    out = np.array([oracle_mod.kmc_network(p, start, kr, i)[0] for i in range(200)])
    third = 3 - pair[0] - pair[1]
    assert np.all(out[:, other] - out[:, small] == c) and not out[:, third].any()
    Xf = X0 / (1.0 + kX0dt) if c == 0 else c * X0 / ((X0 + c) * np.exp(k * c * p.dt) - X0)
    rel = (out[:, small].mean() - Xf) / Xf
    pred = _leap_bias(eps, X0, Xf, c)
    se = out[:, small].std() / Xf / np.sqrt(len(out))
    assert abs(rel - pred) <= 4 * se + eps ** 2, (rel, pred, se)
    # a leap twice as long (g = 1 instead of 2) would double the bias
    assert abs(rel - 2 * pred) > 4 * se + eps ** 2


def test_ion_ion_recombination_runs_in_cells_without_electrons(oracle_mod):
    """Through the grid entry (beta_np / dV): cells with no electrons but
    ions of both signs recombine with the master equation's distribution;
    cells holding ions of one sign only do nothing, and with beta = 0 no
    ion-only cell fires."""
    n = 32
    ph = synth.physics_small(n)
    dV = synth.cell_size(ph) ** 3
    k = 0.05 / ph["dt"]
    ph["beta_np"] = k * dV
    p = oracle_mod.make_params(ph, seed=4)
    nc = n ** 3
    Xe = np.zeros(nc, np.int64)
    Npos = np.full(nc, 3, np.int64)
    Nneg = np.full(nc, 7, np.int64)
    Nneg[::17] = 0                                                 # one sign only
    E = [np.zeros(nc)] * 3
    from oracle import stages
    ion, att, ph_, ep, npr = stages.kmc(p, Xe, E, Npos, Nneg)
    assert not ion.any() and not att.any() and not ph_.any() and not ep.any()
    assert not npr[::17].any()
    both = np.ones(nc, bool)
    both[::17] = False
    fin = np.stack([Xe, Npos - npr, Nneg - npr], axis=1)[both]
    states, P = _master_equation((0, 3, 7), np.array(_kr(k_np=k)) * (p.dt / ph["dt"]), p.dt)
    stat, crit = _chi2_against(fin, states, P)
    assert stat < crit, (stat, crit)
    # beta = 0: ion-only cells are skipped
    p0 = oracle_mod.make_params(dict(ph, beta_np=0.0), seed=4)
    assert not any(f.any() for f in stages.kmc(p0, Xe, E, Npos, Nneg))


def test_beta_zero_gives_the_first_order_network(oracle_mod):
    """With beta_ep = beta_np = 0 the ion counts do not enter: the firings
    of a cell are those of the single-cell entry that knows no ions."""
    n = 12
    ph = synth.physics_small(n)
    p = oracle_mod.make_params(ph, seed=9)
    rng = np.random.default_rng(1)
    nc = n ** 3
    Xe = rng.integers(0, 10 ** 5, nc).astype(np.int64)
    E = [rng.normal(0, 4e6, nc) for _ in range(3)]
    Npos = rng.integers(0, 10 ** 6, nc).astype(np.int64)
    Nneg = rng.integers(0, 10 ** 6, nc).astype(np.int64)
    from oracle import stages
    f_ions = stages.kmc(p, Xe, E, Npos, Nneg)
    f_none = stages.kmc(p, Xe, E)
    for a, b in zip(f_ions, f_none):
        assert np.array_equal(a, b)
    assert not f_ions[3].any() and not f_ions[4].any() and f_ions[0].sum() > 0


@pytest.mark.parametrize("semi", [False, True])
def test_whole_steps_with_recombination_conserve_charge(oracle_mod, semi):
    """Whole steps with the air coefficients of Sec. 5.1 and quasi-neutral
    ions (plus a negative-ion background): both recombinations fire, the net
    charge changes only by the electrons absorbed at the walls, counts stay
    non-negative."""
    from oracle import semi_implicit as si
    from oracle import stages
    n = 16
    ph = synth.with_recombination(dict(synth.physics_small(n), dt=5e-12, photon_ratio=0.06))
    st = synth.blob_state(ph, seed=3, sigma=1.2e-3, peak=5e18, zfrac=0.5)
    p = oracle_mod.make_params(ph, seed=8, step=0)
    S = oracle_mod.canonical(p, st)
    n3 = n ** 3
    cnt = np.bincount(S["cell"], weights=S["w"].astype(np.float64), minlength=n3).astype(np.int64)
    rng = np.random.default_rng(2)
    S["Nneg"] = rng.integers(10 ** 7, 10 ** 8, n3).astype(np.int64)
    S["Npos"] = cnt + S["Nneg"]
    E = synth.random_field(ph, seed=3, amp=2e6, base=4e6)
    q0 = int(S["Npos"].sum() - S["Nneg"].sum()) - int(S["w"].astype(np.int64).sum())
    fired_ep = fired_np = 0
    for k in range(2):
        p = oracle_mod.make_params(ph, seed=8, step=k)
        S, info = si.step(p, ph, S) if semi else stages.step(p, S, E)
        q1 = int(S["Npos"].sum() - S["Nneg"].sum()) - int(S["w"].astype(np.int64).sum())
        assert q1 - q0 == info["outflow"], (q1 - q0, info["outflow"])
        q0 = q1
        assert np.all(S["Npos"] >= 0) and np.all(S["Nneg"] >= 0) and np.all(S["w"] > 0)
        fired_ep += int(info["n_ep"].sum())
        fired_np += int(info["n_np"].sum())
    assert fired_ep > 0 and fired_np > 0

