"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: an exact
invariant of the discrete scheme (mass conservation, the volume budget, lake at
rest, mirror symmetry), a closed-form solution of the PDEs (Thacker's bowl, the
friction ODE, the linear standing wave and its discrete dispersion relation) or
a physical bound (radiation reflection, nested vs fine-grid solution).
"""
import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import numpy as np
import pytest

G = 9.81


def single(nx, ny, dx, h, n=0.0, bc=(0, 0, 0, 0)):
    blk = dict(level=1, parent=-1, nx=nx, ny=ny, i0=0, j0=0, dx=dx, bc=bc)
    hh = np.broadcast_to(np.asarray(h, np.float64), (ny, nx)).copy()
    nn = np.broadcast_to(np.asarray(n, np.float32), (ny, nx)).copy()
    return blk, hh, nn


def centres(n, dx):
    return (np.arange(n) + 0.5) * dx


# ----------------------------------------------------------------------------- Eq. 1
def test_closed_basin_mass_conservation(oracle_mod):
    """Walls, no drying: the flux differences of Eq. 1 telescope, so sum(eta) is
    constant to rounding over 10^4 steps (with friction and advection on)."""
    nx, ny, dx = 64, 48, 2000.0
    x, y = centres(nx, dx), centres(ny, dx)
    h = 200.0 + 100.0 * np.sin(x[None, :] / 9e3) * np.cos(y[:, None] / 7e3)
    blk, hh, nn = single(nx, ny, dx, h, n=0.025)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=10.0)
    dz = 3.0 * np.exp(-((x[None, :] - 40e3) ** 2 + (y[:, None] - 50e3) ** 2) / (2 * 8e3**2))
    o.set_initial_uplift(0, dz)
    e0, _, _ = o.get_state(0)
    s0, a0 = e0.sum(), np.abs(e0).sum()
    v0 = o.budget(0)["volume"]
    o.step(10000)
    e1, _, _ = o.get_state(0)
    b = o.budget(0)
    assert np.abs(e1).max() > 1e-3  # the wave is still there
    assert abs(e1.sum() - s0) <= 1e-12 * a0
    assert abs(b["volume"] - v0) <= 1e-13 * v0
    assert b["outflow"] == 0.0 and b["clip"] == 0.0 and b["ring"] == 0.0


def test_budget_closes_with_drying_and_radiation(oracle_mod):
    """Beach that dries and floods plus an open west edge: V(t) = V0 - outflow + clip."""
    nx, ny, dx = 80, 40, 500.0
    x = centres(nx, dx)
    prof = np.where(x < 25e3, 60.0, 60.0 - (x - 25e3) * 0.006)  # beach rising to land
    h = np.tile(prof, (ny, 1))
    blk, hh, nn = single(nx, ny, dx, h, n=0.03, bc=(1, 0, 0, 0))
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=2.0)
    y = centres(ny, dx)
    o.set_initial_uplift(0, 4.0 * np.exp(-((x[None, :] - 20e3) ** 2) / (2 * 3e3**2)) +
                         0 * y[:, None])
    v0 = o.budget(0)["volume"]
    wet0 = hh + o.get_state(0)[0] > 1e-3
    flooded = np.zeros_like(wet0)
    for _ in range(30):
        o.step(100)
        flooded |= (hh + o.get_state(0)[0] > 1e-3) & ~wet0
    b = o.budget(0)
    assert b["outflow"] != 0 and flooded.sum() > 40  # the shore moved
    assert abs(b["volume"] - (v0 - b["outflow"] + b["clip"])) <= 1e-12 * v0


# ----------------------------------------------------------------------- Eqs. 2-3 at rest
def _rest_hierarchy(scen):
    sc = scen.coastal_hierarchy("rest", 11, (60, 54, 810.0), [(1, 36, 36), (1, 27, 27)],
                                dt=0.5, steps=0, shelf_w=8e3, slope_w=10e3, wiggle=1e3,
                                coast_frac=0.6, land_frac=0.4, relief_amp=3.0)
    return sc


def test_lake_at_rest_nested_bitwise(oracle_mod, nest_feedback=0, nest_flux=0, steps=10000):
    """eta = 0 on sea, -h on land, no flux, over rough bathymetry with land and three
    nested levels: every term of Eqs. 2-3 vanishes, bitwise, for 10^4 steps."""
    from paper_2408_07609_gb300 import scenarios as S

    sc = _rest_hierarchy(S)
    assert any((h <= 0).any() for h in sc.bathy) and any((h > 0).any() for h in sc.bathy)
    o = oracle_mod.Oracle(sc.blocks, sc.bathy, sc.manning, sc.dt, nest_feedback=nest_feedback,
                          nest_flux=nest_flux)
    o.step(steps)
    for k in range(len(sc.blocks)):
        e, M, N = o.get_state(k)
        rest = np.where(sc.bathy[k] > 0, 0.0, -sc.bathy[k])
        assert np.array_equal(e, rest)
        assert not M.any() and not N.any()
        b = o.budget(k)
        assert b["clip"] == 0 and b["outflow"] == 0 and b["ring"] == 0


# ------------------------------------------------------------------ linear standing wave
@pytest.mark.parametrize("cfl", [0.3, 0.7])
def test_standing_wave_discrete_period(oracle_mod, cfl):
    """Flat closed basin, mode cos(pi x / L), amplitude 1e-6 h, no friction. The linear
    leap-frog staggered scheme has the exact discrete dispersion relation
    sin(w dt / 2) = (c dt / dx) sin(k dx / 2); the measured period must match it to
    1e-5 (and differs visibly from the continuum 2L/c at coarse resolution)."""
    nx, ny, dx, h = 24, 4, 1000.0, 100.0
    c = math.sqrt(G * h)
    dt = cfl * dx / c
    blk, hh, nn = single(nx, ny, dx, h)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=dt)
    L = nx * dx
    k = math.pi / L
    x = centres(nx, dx)
    a = 1e-6 * h
    o.set_initial_uplift(0, np.tile(a * np.cos(k * x), (ny, 1)))
    w = 2.0 / dt * math.asin(c * dt / dx * math.sin(k * dx / 2))
    T_disc, T_cont = 2 * math.pi / w, 2 * L / c
    nsteps = int(2.5 * T_disc / dt)
    series = []
    for _ in range(nsteps):
        o.step(1)
        series.append(o.get_state(0)[0][1, 0])
    s = np.array(series)
    # cos(w dt) from the two-step recurrence where |eta| is not small
    mid = s[1:-1]
    sel = np.abs(mid) > 0.5 * a
    cos_wdt = np.median((s[2:][sel] + s[:-2][sel]) / (2 * mid[sel]))
    T_fit = 2 * math.pi * dt / math.acos(cos_wdt)
    assert abs(T_fit - T_disc) <= 1e-5 * T_disc
    assert abs(T_disc - T_cont) > 1e-5 * T_cont  # the discrete period is what is pinned
    # amplitude neither grows nor decays (neutral leap-frog)
    assert abs(np.abs(s).max() - a) < 0.02 * a


# ---------------------------------------------------------------- Thacker parabolic bowl
def thacker(r, t, h0, a, r0):
    A = (a**4 - r0**4) / (a**4 + r0**4)
    w = math.sqrt(8 * G * h0) / a
    cw = math.cos(w * t)
    return h0 * (math.sqrt(1 - A * A) / (1 - A * cw) - 1 -
                 (r * r / (a * a)) * ((1 - A * A) / (1 - A * cw) ** 2 - 1)), w


def run_thacker(oracle_mod, dx, h0=50.0, a=80e3, r0=70e3, dt=5.0):
    half = 100e3  # the shoreline swings between r0 = 70 km and 91.4 km
    n = int(round(2 * half / dx))
    x = centres(n, dx) - half
    r = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2)
    h = h0 * (1 - r**2 / a**2)
    blk, hh, nn = single(n, n, dx, h)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=dt)
    eta0, w = thacker(r, 0.0, h0, a, r0)
    o.set_initial_uplift(0, eta0)
    T = 2 * math.pi / w
    errs = []
    done = 0
    for frac in (0.5, 1.0):
        target = int(round(frac * T / dt))
        o.step(target - done)
        done = target
        ex, _ = thacker(r, done * dt, h0, a, r0)
        e, _, _ = o.get_state(0)
        both = (h + ex > 0) & (h + e > 1e-3)
        errs.append(np.abs(e - ex)[both].mean() / h0)
    assert o.budget(0)["clip"] == 0.0  # the outflow limit keeps every cell non-negative
    return errs


def test_thacker_parabolic_bowl(oracle_mod):
    """Thacker (1981) analytic moving-shoreline solution of the nonlinear SWE (Eqs. 1-3
    with n = 0) tests advection, the wet/dry front and the depth terms together.
    A = (a^4 - r0^4)/(a^4 + r0^4) = 0.26: the shoreline moves 21 km each half period."""
    e1 = run_thacker(oracle_mod, 1000.0)
    e2 = run_thacker(oracle_mod, 500.0)
    for e in e1 + e2:
        assert e <= 0.03
    # refinement lowers the error
    assert e2[0] < 0.8 * e1[0] and e2[1] < 0.8 * e1[1]


# -------------------------------------------------------------------- mirror symmetry
def test_mirror_and_transpose_symmetry_bitwise(oracle_mod):
    """Symmetric square basin with a symmetric island (drying on), centred source:
    x-mirror, y-mirror and transposition are exact symmetries of Eqs. 1-3 and of the
    scheme's operation order, so they hold bitwise."""
    n, dx = 60, 1000.0
    x = centres(n, dx) - n * dx / 2
    r = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2)
    h = 80.0 - 95.0 * np.exp(-(r / 6e3) ** 2)  # island in the middle
    blk, hh, nn = single(n, n, dx, h, n=0.03)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=5.0)
    ring = 2.5 * np.exp(-((r - 15e3) / 4e3) ** 2)
    o.set_initial_uplift(0, ring)
    wet0 = hh + o.get_state(0)[0] > 1e-3
    flips = 0
    for _ in range(4):
        o.step(150)
        e, M, N = o.get_state(0)
        assert np.array_equal(e, e[:, ::-1])
        assert np.array_equal(e, e[::-1, :])
        assert np.array_equal(e, e.T)
        assert np.array_equal(M, -M[:, ::-1])
        assert np.array_equal(N, -N[::-1, :])
        assert np.array_equal(M, N.T)
        flips += ((hh + e > 1e-3) != wet0).sum()
    assert flips > 0  # the island's shore flooded and dried


# ------------------------------------------------------------------------- friction
def test_friction_matches_manning_ode(oracle_mod):
    """Uniform flux over a flat bed, far from the walls: Eq. 2 reduces to
    dM/dt = -g n^2 M|M| / h^(7/3), solved by M0 / (1 + k M0 t). The semi-implicit
    scheme is first order in time: the error halves with dt."""
    nx, ny, dx, h, nman, M0 = 200, 20, 500.0, 5.0, 0.03, 2.0
    k = G * nman**2 / h ** (7.0 / 3.0)
    errs = []
    for dt in (4.0, 2.0):
        blk, hh, nn = single(nx, ny, dx, h, n=nman)
        o = oracle_mod.Oracle([blk], [hh], [nn], dt=dt)
        M = np.full((ny, nx + 1), M0)
        M[:, 0] = M[:, -1] = 0.0
        o.set_state(0, eta=np.zeros((ny, nx)), M=M, N=np.zeros((ny + 1, nx)))
        steps = int(round(40.0 / dt))
        o.step(steps)
        _, M1, _ = o.get_state(0)
        exact = M0 / (1 + k * M0 * steps * dt)
        mid = M1[:, nx // 2 - 5: nx // 2 + 5]
        assert np.all(mid == mid[0, 0])  # untouched by the walls
        errs.append(abs(mid[0, 0] - exact) / exact)
    assert errs[0] < 2e-3
    assert 1.6 < errs[0] / errs[1] < 2.4


# ------------------------------------------------------- advection: time level of the depth
def stretching_flow(oracle_mod, along_x, dt, steps, dx=100.0, h=10.0, a0=1e-3, b0=5.0, n=200):
    """Uniform stretching flow over a flat, frictionless bed: the flux grows linearly
    along the flow, q(s) = a s + b (s = f dx at face f), the depth D is uniform and falls
    as dD/dt = -a, so the water surface stays flat and the pressure term of Eqs. 2-3
    vanishes; only the advective term d(q^2/D)/ds acts. The walls disturb the flow only
    within two faces per step of themselves (the stencil's reach). Returns the oracle's
    (a, b, D) after `steps` steps, fitted on the undisturbed middle faces, with the
    largest deviation from the linear profile."""
    ny = 3
    nx_, ny_ = (n, ny) if along_x else (ny, n)
    blk, hh, nn = single(nx_, ny_, dx, h)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=dt)
    q = a0 * np.arange(n + 1) * dx + b0
    q[0] = q[n] = 0.0  # walls
    if along_x:
        o.set_state(0, eta=np.zeros((ny, n)), M=np.tile(q, (ny, 1)), N=np.zeros((ny + 1, n)))
    else:
        o.set_state(0, eta=np.zeros((n, ny)), M=np.zeros((n, ny + 1)),
                    N=np.tile(q[:, None], (1, ny)))
    o.step(steps)
    e, M, N = o.get_state(0)
    if along_x:
        qf, ec, across = M[1], e[1], N
    else:
        qf, ec, across = N[:, 1], e[:, 1], M
    lo, hi = 2 * steps + 4, n - 2 * steps - 4
    s = np.arange(lo, hi + 1) * dx
    a, b = np.polyfit(s, qf[lo:hi + 1], 1)
    dev = np.abs(qf[lo:hi + 1] - (a * s + b)).max()
    D = h + ec[lo:hi]
    assert not across.any()  # the flow stays one-dimensional
    assert np.ptp(D) <= 1e-12 * h  # and the surface flat
    return a, b, D.mean(), dev


def test_advective_depth_is_the_new_level(oracle_mod):
    """R2/R3: the advective fluxes M^2/D, M Nbar/D (N^2/D, N Mbar/D) divide by the face
    depth of the new level eta^{n+1}, the level at t^{n+1/2} where the leap-frog
    momentum update of Eqs. 2-3 is centred (Sec. II-A) and which its pressure term
    already uses. On the stretching flow of `stretching_flow` (walls far away, q > 0 so
    the upwind difference takes the lower face) one step is, in closed form, with
    D' = D - dt a the new depth:
        a' = a (1 - 2 dt a / D'),   b' = b - dt a (2 b - a dx) / D'
    (the a dx term is the upwind difference's own diffusion), and the oracle must follow
    it to rounding in both directions. A depth from the old level eta^n gives
    a' = a (1 - 2 dt a / D) instead. As dt -> 0 the recursion tends to the exact
    solution of Eqs. 1-2 for this flow, a / D^2 constant (D(t) = D0 / (1 + a0 t / D0)),
    which the oracle approaches at first order."""
    dx, h, a0, b0, dt, K = 100.0, 10.0, 1e-3, 5.0, 2.0, 20
    a, b, D = a0, b0, h
    for _ in range(K):
        D1 = D - dt * a
        a, b, D = a * (1 - 2 * dt * a / D1), b - dt * a * (2 * b - a * dx) / D1, D1
    a_old, D_old = a0, h
    for _ in range(K):  # the old-level reading, for scale
        a_old, D_old = a_old * (1 - 2 * dt * a_old / D_old), D_old - dt * a_old
    assert abs(a - a_old) > 1e-7 * a  # the two readings differ far above rounding
    for along_x in (True, False):
        ga, gb, gD, dev = stretching_flow(oracle_mod, along_x, dt, K, dx, h, a0, b0)
        assert dev <= 1e-12 * b0
        assert abs(ga - a) <= 1e-11 * a, (along_x, ga, a, a_old)
        assert abs(gb - b) <= 1e-11 * b, (along_x, gb, b)
        assert abs(gD - D) <= 1e-12 * h
    # first order towards the exact solution of the PDE over t = 40 s
    T, errs = 40.0, []
    exact_a = a0 / (1 + a0 * T / h) ** 2
    for dt in (2.0, 1.0):
        ga = stretching_flow(oracle_mod, True, dt, int(round(T / dt)), dx, h, a0, b0)[0]
        errs.append(abs(ga - exact_a) / exact_a)
    assert errs[0] < 1e-3 and 1.8 < errs[0] / errs[1] < 2.2


# --------------------------------------------------------------- the friction term's D^(7/3)
def test_cube_root_is_within_four_ulp(oracle_mod):
    """Eq. 2's friction divides by D^(7/3) = D^2 cbrt(D). The oracle takes the cube root
    by a stated Newton iteration (so that a binary64 implementation with the same
    operations rounds identically); it must be within 4 ulp of the correctly rounded cube
    root over the depths a model meets (1 mm to 100 km), exact on exact cubes, and
    monotone."""
    L = oracle_mod.lib()
    rng = np.random.default_rng(11)
    xs = np.exp(rng.uniform(np.log(1e-3), np.log(1e5), 50000))
    xs = np.concatenate([xs, [1e-3, 0.5, 1.0, 2.0, 4.0, 7000.0, 1e5]])
    got = np.array([L.orc_cube_root(float(x)) for x in xs])
    ref = np.cbrt(xs)
    assert (np.abs(got - ref) / np.spacing(ref)).max() <= 4.0
    for k in (1, 2, 3, 5, 10, 17, 100):
        assert L.orc_cube_root(float(k) ** 3) == float(k)
    srt = np.sort(xs)
    cr = np.array([L.orc_cube_root(float(x)) for x in srt])
    assert np.all(np.diff(cr) >= 0)


# ------------------------------------------------------------------------- radiation
def test_radiation_west_edge_absorbs(oracle_mod):
    """A left-going linear long wave (M = -c eta) leaves through the radiation edge;
    the energy left in the channel afterwards is < 2 % of the initial energy."""
    nx, ny, dx, h = 400, 4, 1000.0, 100.0
    c = math.sqrt(G * h)
    dt = 10.0
    blk, hh, nn = single(nx, ny, dx, h, bc=(1, 0, 0, 0))
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=dt)
    x = centres(nx, dx)
    xf = np.arange(nx + 1) * dx
    amp = 0.05
    eta = np.tile(amp * np.exp(-((x - 200e3) / 15e3) ** 2), (ny, 1))
    M = np.tile(-c * amp * np.exp(-((xf - 200e3) / 15e3) ** 2), (ny, 1))
    M[:, -1] = 0.0
    o.set_state(0, eta=eta, M=M, N=np.zeros((ny + 1, nx)))

    def energy():
        e, M, N = o.get_state(0)
        return 0.5 * G * (e**2).sum() + 0.5 * ((M**2).sum() + (N**2).sum()) / h

    E0 = energy()
    o.step(int(round(320e3 / c / dt)))
    assert energy() < 0.02 * E0


# ------------------------------------------------------------------------- nesting
def nested_flat(dxp=300.0, h=50.0, npx=90, npy=30, cx=30, cw=30, cy=6, ch=18, bc=(1, 1, 0, 0)):
    blocks = [dict(level=1, parent=-1, nx=npx, ny=npy, i0=0, j0=0, dx=dxp, bc=bc),
              dict(level=2, parent=0, nx=3 * cw, ny=3 * ch, i0=cx, j0=cy, dx=dxp / 3, bc=(0,) * 4)]
    bathy = [np.full((npy, npx), h), np.full((3 * ch, 3 * cw), h)]
    man = [np.zeros((npy, npx), np.float32), np.zeros((3 * ch, 3 * cw), np.float32)]
    return blocks, bathy, man


def test_nest_constant_field_ring_average(oracle_mod):
    """A constant child field averages (Listing 5: sum of 9 times 1/9) to itself within
    one ulp on the parent's ring cells, and inner parent cells keep their own value."""
    blocks, bathy, man = nested_flat()
    o = oracle_mod.Oracle(blocks, bathy, man, dt=2.0)
    cval = 0.123456789
    o.set_state(1, eta=np.full((54, 90), cval))
    o.step(1)
    e, _, _ = o.get_state(0)
    I0, J0, a, b = 30, 6, 30, 18
    ring = np.zeros_like(e, bool)
    ring[J0:J0 + b, I0:I0 + a] = True
    ring[J0 + 1:J0 + b - 1, I0 + 1:I0 + a - 1] = False
    assert np.all(np.abs(e[ring] - cval) <= np.spacing(cval))
    assert np.all(e[J0 + 1:J0 + b - 1, I0 + 1:I0 + a - 1] == 0.0)
    assert o.budget(0)["ring"] > 0


def test_nest_edge_flux_reproduces_linear_profile(oracle_mod):
    """Steady shear flow M(y) = a + b y over a flat bed (no friction, N = 0): the parent
    keeps it exactly, and linear interpolation along a child edge must reproduce the
    straight line at every fine face centre away from the clamped segment ends."""
    blocks, bathy, man = nested_flat(bc=(0, 0, 0, 0))
    o = oracle_mod.Oracle(blocks, bathy, man, dt=2.0)
    dxp = blocks[0]["dx"]
    yp = centres(30, dxp)
    Mp = np.tile((0.3 + 2e-5 * yp)[:, None], (1, 91))
    Mp[:, 0] = Mp[:, -1] = 0.0
    o.set_state(0, M=Mp)
    o.step(1)
    _, Mc, _ = o.get_state(1)
    J0 = blocks[1]["j0"]
    yc = J0 * dxp + centres(54, dxp / 3)
    want = 0.3 + 2e-5 * yc
    for f in (0, 90):  # west and east edges
        got = Mc[3:-3, f]
        assert np.allclose(got, want[3:-3], rtol=1e-14, atol=0)
        assert not np.allclose(Mc[3:-3, f], np.repeat(Mp[J0 + 1:J0 + 17, 31], 3), rtol=1e-9)


def test_nested_budget_closes(oracle_mod, nest_feedback=0, nest_flux=0):
    """With nesting, each block's budget closes: V = V0 - outflow + clip + ring."""
    from paper_2408_07609_gb300 import scenarios as S

    sc = S.coastal_hierarchy("b", 5, (60, 54, 810.0), [(1, 36, 36), (1, 27, 27)], dt=0.5,
                             steps=0, shelf_w=8e3, slope_w=10e3, wiggle=1e3, coast_frac=0.6,
                             land_frac=0.4, source=dict(kind="gauss", sigma=4e3, peak=2.0))
    o = oracle_mod.Oracle(sc.blocks, sc.bathy, sc.manning, sc.dt, nest_feedback=nest_feedback,
                          nest_flux=nest_flux)
    for k, dz in enumerate(sc.uplift):
        if dz is not None:
            o.set_initial_uplift(k, dz)
    v0 = [o.budget(k)["volume"] for k in range(3)]
    o.step(2000)
    for k in range(3):
        b = o.budget(k)
        assert abs(b["volume"] - (v0[k] - b["outflow"] + b["clip"] + b["ring"])) <= 1e-12 * v0[k]
    assert o.budget(1)["outflow"] != 0 and o.budget(0)["ring"] != 0


def nested_vs_fine(oracle_mod, nest_feedback=0, nest_flux=0):
    """Largest |eta| difference, inside the patch, between a long plane wave crossing a
    flat nested patch and the same wave on one grid at the child's resolution; and the
    wave's amplitude."""
    dxp, h, amp = 300.0, 50.0, 0.05
    npx, npy = 150, 30
    blocks, bathy, man = nested_flat(dxp, h, npx=npx, npy=npy, cx=60, cw=30, cy=6, ch=18,
                                     bc=(1, 1, 0, 0))
    dt = 2.0
    c = math.sqrt(G * h)
    lam = 12e3
    x0 = 9e3

    def wave(x):
        return amp * np.exp(-((x - x0) / (lam / 4)) ** 2)

    o = oracle_mod.Oracle(blocks, bathy, man, dt=dt, nest_feedback=nest_feedback,
                          nest_flux=nest_flux)
    xp = centres(npx, dxp)
    xfp = np.arange(npx + 1) * dxp
    o.set_state(0, eta=np.tile(wave(xp), (npy, 1)), M=np.tile(c * wave(xfp), (npy, 1)))
    xc = 60 * dxp + centres(90, dxp / 3)
    xfc = 60 * dxp + np.arange(91) * dxp / 3
    o.set_state(1, eta=np.tile(wave(xc), (54, 1)), M=np.tile(c * wave(xfc), (54, 1)))
    blk, hh, nn = single(3 * npx, 3 * npy, dxp / 3, h, bc=(1, 1, 0, 0))
    f = oracle_mod.Oracle([blk], [hh], [nn], dt=dt)
    xf = centres(3 * npx, dxp / 3)
    xff = np.arange(3 * npx + 1) * dxp / 3
    f.set_state(0, eta=np.tile(wave(xf), (3 * npy, 1)), M=np.tile(c * wave(xff), (3 * npy, 1)))
    worst = 0.0
    for _ in range(10):
        o.step(100)
        f.step(100)
        ec = o.get_state(1)[0]
        ef = f.get_state(0)[0][18:18 + 54, 180:180 + 90]
        worst = max(worst, np.abs(ec - ef).max())
    return worst, amp


def test_nested_plane_wave_matches_fine_grid(oracle_mod):
    """A long plane wave crossing a flat nested patch: inside the patch the nested
    solution (coarse flux interpolated in, 3x3 mean fed back) stays within 2 % of the
    amplitude of a single grid at the child's resolution everywhere."""
    worst, amp = nested_vs_fine(oracle_mod)
    assert worst <= 0.02 * amp


# ------------------------------------ nesting options: full feedback (R8), constant flux (R7)
@pytest.mark.parametrize("fb,fl", [(1, 0), (0, 1), (1, 1)])
def test_lake_at_rest_nested_bitwise_with_options(oracle_mod, fb, fl):
    test_lake_at_rest_nested_bitwise(oracle_mod, nest_feedback=fb, nest_flux=fl, steps=2000)


@pytest.mark.parametrize("fb,fl", [(1, 0), (0, 1), (1, 1)])
def test_nested_budget_closes_with_options(oracle_mod, fb, fl):
    test_nested_budget_closes(oracle_mod, nest_feedback=fb, nest_flux=fl)


@pytest.mark.parametrize("fb,fl", [(1, 0), (0, 1), (1, 1)])
def test_nested_plane_wave_matches_fine_grid_with_options(oracle_mod, fb, fl):
    """Every nesting option keeps the nested wave within 2 % of the fine-grid wave."""
    worst, amp = nested_vs_fine(oracle_mod, nest_feedback=fb, nest_flux=fl)
    assert worst <= 0.02 * amp


def test_full_feedback_sets_every_covered_cell_to_the_child_mean(oracle_mod):
    """Full two-way nesting. (i) A constant child field averages to itself within one ulp
    on every covered parent cell, not just the ring. (ii) A pulse over a flat two-level
    nest: after each step every covered parent cell equals the mean of its 3x3 child
    cells (all wet; with two levels the child's levels after the step are the values
    that were averaged) to rounding, while with ring feedback the inner cells keep
    values of their own."""
    blocks, bathy, man = nested_flat()
    I0, J0, a, b = 30, 6, 30, 18
    o = oracle_mod.Oracle(blocks, bathy, man, dt=2.0, nest_feedback=oracle_mod.NEST_FULL)
    cval = 0.123456789
    o.set_state(1, eta=np.full((54, 90), cval))
    o.step(1)
    e = o.get_state(0)[0]
    assert np.all(np.abs(e[J0:J0 + b, I0:I0 + a] - cval) <= np.spacing(cval))
    assert o.budget(0)["ring"] > 0

    def pulse(x, y, cx, cy):
        return 0.2 * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * 1500.0 ** 2))

    dxp = blocks[0]["dx"]
    xp, yp = np.meshgrid(centres(90, dxp), centres(30, dxp))
    xc, yc = np.meshgrid(I0 * dxp + centres(90, dxp / 3), J0 * dxp + centres(54, dxp / 3))
    cx, cy = (I0 + 12) * dxp, (J0 + 7) * dxp
    gaps = {}
    for fb in (oracle_mod.NEST_RING, oracle_mod.NEST_FULL):
        o = oracle_mod.Oracle(blocks, bathy, man, dt=2.0, nest_feedback=fb)
        o.set_state(0, eta=pulse(xp, yp, cx, cy))
        o.set_state(1, eta=pulse(xc, yc, cx, cy))
        gap = 0.0
        for _ in range(20):
            o.step(1)
            ep, ec = o.get_state(0)[0], o.get_state(1)[0]
            mean = ec.reshape(b, 3, a, 3).mean(axis=(1, 3))
            cover = ep[J0:J0 + b, I0:I0 + a]
            if fb == oracle_mod.NEST_FULL:
                assert np.all(np.abs(cover - mean) <= 4 * np.spacing(np.abs(mean).max()))
            gap = max(gap, np.abs(cover - mean)[1:-1, 1:-1].max())
        gaps[fb] = gap
    assert gaps[oracle_mod.NEST_RING] > 1e-6  # the ring option leaves the inner cells alone


def test_constant_flux_gives_each_fine_face_its_coarse_face(oracle_mod):
    """Piecewise-constant coarse-to-fine flux on steady shear flow M(y) = a + b y: each
    fine face of a child edge carries exactly the parent flux of the coarse face it lies
    on, so the edge passes exactly the coarse discharge (3 fine faces of dx/3 each)."""
    blocks, bathy, man = nested_flat(bc=(0, 0, 0, 0))
    o = oracle_mod.Oracle(blocks, bathy, man, dt=2.0, nest_flux=oracle_mod.FLUX_CONSTANT)
    dxp = blocks[0]["dx"]
    yp = centres(30, dxp)
    Mp = np.tile((0.3 + 2e-5 * yp)[:, None], (1, 91))
    Mp[:, 0] = Mp[:, -1] = 0.0
    o.set_state(0, M=Mp)
    o.step(1)
    P = o.get_state(0)[1]
    Mc = o.get_state(1)[1]
    I0, J0 = blocks[1]["i0"], blocks[1]["j0"]
    for f, F in ((0, I0), (90, I0 + 30)):
        coarse = P[J0:J0 + 18, F]
        assert np.array_equal(Mc[:, f], np.repeat(coarse, 3))
        fine_q = Mc[:, f].reshape(18, 3).sum(axis=1) * (dxp / 3)
        assert np.allclose(fine_q, coarse * dxp, rtol=1e-15, atol=0)
    assert not np.allclose(np.diff(Mc[3:-3, 0]), 0.0)  # the profile is really sheared


# ------------------------------------------------------------------------- outputs (R9)
def test_max_and_arrival_are_functions_of_history(oracle_mod):
    from paper_2408_07609_gb300 import scenarios as S

    sc = S.config1(nx=48, ny=40)
    sc.uplift[0][5, 7] = sc.arrival_thr  # a cell exactly at the threshold arrives at t = 0
    o = oracle_mod.from_scenario(sc)
    h = sc.bathy[0]
    e0 = o.get_state(0)[0]
    hist = [e0]
    for _ in range(120):
        o.step(1)
        hist.append(o.get_state(0)[0])
    H = np.array(hist)
    wet = (h[None] + H) > sc.dry_eps
    masked = np.where(wet, H, -np.inf)
    emax = masked.max(axis=0)
    never = ~wet.any(axis=0)
    got = o.max_height(0)
    assert np.array_equal(np.isnan(got), never)
    assert np.array_equal(got[~never], emax[~never])
    md = o.max_depth(0)
    assert np.array_equal(md[~never], h[~never] + emax[~never]) and np.all(md[never] == 0)
    run = np.maximum.accumulate(masked, axis=0)
    reached = run >= sc.arrival_thr
    first = np.where(reached.any(axis=0), reached.argmax(axis=0), -1)
    exp_t = np.where(first >= 0, first * sc.dt, -1.0)
    assert np.array_equal(o.arrival_time(0), exp_t)
    assert (first > 0).sum() > 100 and exp_t[5, 7] == 0.0


# ------------------------------------------------------------------------- validation
def test_cfl_and_nesting_rejected(oracle_mod):
    blk, hh, nn = single(30, 30, 100.0, 1000.0)
    with pytest.raises(oracle_mod.OracleError) as ei:
        oracle_mod.Oracle([blk], [hh], [nn], dt=1.0)  # 100 m/s < sqrt(2 g 1000) = 140
    assert ei.value.code == -2
    oracle_mod.Oracle([blk], [hh], [nn], dt=0.7)
    blocks, bathy, man = nested_flat()
    bad = [dict(b) for b in blocks]
    bad[1]["i0"] = 2  # closer than 3 parent cells to the edge
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(bad, bathy, man, dt=2.0)
    bad = [dict(b) for b in blocks]
    bad[1]["dx"] = 99.0
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(bad, bathy, man, dt=2.0)


# ---------------------------------------------------------------- R11 max velocity
def _flat_basin(oracle_mod, nx=64, ny=64, h=8.0, n=0.0, dt=1.0, dx=100.0):
    blk = dict(level=1, parent=-1, nx=nx, ny=ny, i0=0, j0=0, dx=dx, bc=(0, 0, 0, 0))
    bathy = np.full((ny, nx), h)
    man = np.full((ny, nx), n, np.float32)
    return oracle_mod.Oracle([blk], [bathy], [man], dt)


def test_max_velocity_of_uniform_flow_is_exact(oracle_mod):
    """Uniform frictionless flow over a flat bottom is an exact steady solution away from
    the walls: M = 4, N = 3 m^2/s on h = 8 m gives u = 1/2, v = 3/8 and a speed of exactly
    5/8 m/s in every cell the walls have not yet reached (the scheme's stencil spreads
    one cell per step)."""
    o = _flat_basin(oracle_mod)
    nx = ny = 64
    M = np.full((ny, nx + 1), 4.0)
    M[:, 0] = M[:, nx] = 0.0
    N = np.full((ny + 1, nx), 3.0)
    N[0, :] = N[ny, :] = 0.0
    o.set_state(0, eta=np.zeros((ny, nx)), M=M, N=N)
    o.step(10)
    v = o.max_velocity(0)
    core = v[20:44, 20:44]
    assert np.all(core == 0.625)
    e, M1, N1 = o.get_state(0)
    assert np.all(M1[20:44, 20:44] == 4.0) and np.all(e[20:44, 20:44] == 0.0)


def test_max_velocity_averages_the_two_faces_of_a_cell(oracle_mod):
    """Flux fields linear in x and in y, M(f, j) = f / 4 and N(i, g) = g / 8, give the
    cell-centre velocity ((i + 1/2) / 4, (j + 1/2) / 8) / h (closed form of the face
    means): a shifted face index, a dropped 1/2 or a missing depth changes the values.
    Read before any step, so only the current state counts."""
    nx, ny, h = 16, 12, 2.0
    o = _flat_basin(oracle_mod, nx=nx, ny=ny, h=h)
    M = np.tile(np.arange(nx + 1, dtype=float) / 4.0, (ny, 1))
    N = np.tile((np.arange(ny + 1, dtype=float) / 8.0)[:, None], (1, nx))
    o.set_state(0, eta=np.zeros((ny, nx)), M=M, N=N)
    u = np.tile((np.arange(nx) + 0.5) / 4.0, (ny, 1)) / h
    v = np.tile(((np.arange(ny) + 0.5) / 8.0)[:, None], (1, nx)) / h
    assert np.allclose(o.max_velocity(0), np.hypot(u, v), rtol=1e-15, atol=0)
    # with N alone the speed is the y component, exactly
    o.set_state(0, M=np.zeros((ny, nx + 1)))
    assert np.array_equal(o.max_velocity(0), v)


def test_max_velocity_takes_each_face_over_its_own_depth(oracle_mod):
    """R11 divides each face's flux by that face's depth: over a bottom deepening by 1 m a
    cell (h_i = 2 + i, eta = 0) with a uniform x-flux of 1 m^2/s between walls, face f lies
    between depths 1 + f and 2 + f, so its depth is 1.5 + f and the cell-centre speed is
    (1/(1.5 + i) + 1/(2.5 + i))/2, with 0 for a wall face (whose depth is the edge cell's);
    the mean flux over the cell's depth, 1/(2 + i), differs."""
    nx, ny = 12, 3
    blk = dict(level=1, parent=-1, nx=nx, ny=ny, i0=0, j0=0, dx=100.0, bc=(0, 0, 0, 0))
    h = np.tile(2.0 + np.arange(nx, dtype=float), (ny, 1))
    o = oracle_mod.Oracle([blk], [h], [np.zeros((ny, nx), np.float32)], dt=1.0)
    M = np.ones((ny, nx + 1))
    M[:, 0] = M[:, nx] = 0.0
    o.set_state(0, eta=np.zeros((ny, nx)), M=M, N=np.zeros((ny + 1, nx)))
    i = np.arange(nx, dtype=float)
    uw = np.where(i > 0, 1.0 / (1.5 + i), 0.0)
    ue = np.where(i < nx - 1, 1.0 / (2.5 + i), 0.0)
    want = np.tile(0.5 * (uw + ue), (ny, 1))
    got = o.max_velocity(0)
    assert np.allclose(got, want, rtol=1e-15, atol=0)
    assert not np.allclose(got[:, 1:-1], 1.0 / (2.0 + i[1:-1]), rtol=1e-3)


def test_max_velocity_is_zero_at_rest_and_on_dry_land_and_grows_monotonically(oracle_mod):
    """Lake at rest: 0 everywhere. After a source: a running maximum (never decreases
    between reads), positive where the wave passed, 0 on land that never got wet."""
    from paper_2408_07609_gb300 import scenarios as S

    sc = S.config1(nx=96, ny=64, steps=0)
    o = oracle_mod.from_scenario(sc)
    o.set_initial_uplift(0, np.zeros((64, 96)))
    o.step(50)
    assert np.all(o.max_velocity(0) == 0.0)  # lake at rest
    o.set_initial_uplift(0, sc.uplift[0])
    prev = o.max_velocity(0)
    for _ in range(5):
        o.step(40)
        cur = o.max_velocity(0)
        assert np.all(cur >= prev)
        prev = cur
    never_wet = np.isnan(o.max_height(0))
    assert prev.max() > 0.01 and never_wet.any() and np.all(prev[never_wet] == 0.0)


def pulse_nested_vs_fine(oracle_mod, nest_feedback, nest_flux, dxp=300.0, h=50.0, amp=0.1):
    """A Gaussian pulse (sigma 1.5 km) spreads from outside a flat 2-level nest into the
    child (30 x 30 parent cells, dx 100 m) and is compared, every 20 s for 400 s, with
    the same pulse on one grid at 100 m. Returns the largest |eta| differences in the
    child, on the parent cells the child covers (against the fine grid's 3 x 3 means)
    and on the other parent cells, each over the amplitude."""
    npx, npy, I0, J0, cw = 90, 60, 36, 15, 30

    def pulse(x, y):
        return amp * np.exp(-((x - 20 * dxp) ** 2 + (y - 30 * dxp) ** 2) / (2 * 1500.0 ** 2))

    blocks = [dict(level=1, parent=-1, nx=npx, ny=npy, i0=0, j0=0, dx=dxp, bc=(1, 1, 1, 1)),
              dict(level=2, parent=0, nx=3 * cw, ny=3 * cw, i0=I0, j0=J0, dx=dxp / 3,
                   bc=(0,) * 4)]
    bathy = [np.full((npy, npx), h), np.full((3 * cw, 3 * cw), h)]
    man = [np.zeros((npy, npx), np.float32), np.zeros((3 * cw, 3 * cw), np.float32)]
    o = oracle_mod.Oracle(blocks, bathy, man, dt=2.0, nest_feedback=nest_feedback,
                          nest_flux=nest_flux)
    xp, yp = np.meshgrid(centres(npx, dxp), centres(npy, dxp))
    xc, yc = np.meshgrid(I0 * dxp + centres(3 * cw, dxp / 3), J0 * dxp + centres(3 * cw, dxp / 3))
    o.set_state(0, eta=pulse(xp, yp))
    o.set_state(1, eta=pulse(xc, yc))
    blk, hh, nn = single(3 * npx, 3 * npy, dxp / 3, h, bc=(1, 1, 1, 1))
    f = oracle_mod.Oracle([blk], [hh], [nn], dt=2.0)
    xf, yf = np.meshgrid(centres(3 * npx, dxp / 3), centres(3 * npy, dxp / 3))
    f.set_state(0, eta=pulse(xf, yf))
    cov = (slice(J0, J0 + cw), slice(I0, I0 + cw))
    out = np.ones((npy, npx), bool)
    out[cov] = False
    err = np.zeros(3)
    for _ in range(20):
        o.step(10)
        f.step(10)
        ef = f.get_state(0)[0]
        efc = ef.reshape(npy, 3, npx, 3).mean(axis=(1, 3))
        ep, ec = o.get_state(0)[0], o.get_state(1)[0]
        err = np.maximum(err, [np.abs(ec - ef[3 * J0:3 * (J0 + cw), 3 * I0:3 * (I0 + cw)]).max(),
                               np.abs(ep[cov] - efc[cov]).max(), np.abs(ep[out] - efc[out]).max()])
    return err / amp


def test_nested_pulse_vs_fine_grid_for_every_option(oracle_mod):
    """Nested against single-fine-grid accuracy for the four nesting options. Every one
    keeps the child within 1 % of the amplitude; full feedback brings the covered parent
    cells to the child's accuracy (ring feedback leaves them at the coarse grid's); the
    parent cells outside are the coarse grid's own error under every option."""
    e = {(fb, fl): pulse_nested_vs_fine(oracle_mod, fb, fl) for fb in (0, 1) for fl in (0, 1)}
    for v in e.values():
        assert v[0] <= 0.01
    for fl in (0, 1):
        assert e[(1, fl)][1] < 0.85 * e[(0, fl)][1]
        assert e[(1, fl)][1] <= 1.1 * e[(1, fl)][0]
    outside = [v[2] for v in e.values()]
    assert max(outside) - min(outside) <= 1e-3 * max(outside)


def test_outflow_limit_on_a_puddle(oracle_mod):
    """The outflow limit of the wet/dry front (reading R4): a face carries at most a
    quarter of its upwind cell's water per step. A 0.1 m puddle in one cell of flat land
    (ground 1 m above the datum, no friction, dt/dx = 1 s/m, which Eq. 4 allows because
    no cell is sea) sees the front flux g D^2 dt/dx = 0.0981 m^2/s on each of its four
    faces, which the limit cuts to D dx / (4 dt) = 0.025: after one step the four faces
    carry exactly that outward, and after the second mass update the puddle is empty
    and each neighbour holds 0.025 m, with the volume unchanged and no clip."""
    nx = ny = 5
    blk, hh, nn = single(nx, ny, 1.0, -1.0)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=1.0)
    eta = np.full((ny, nx), 1.0)
    eta[2, 2] = 1.1
    o.set_state(0, eta=eta)
    v0 = o.budget(0)["volume"]
    o.step(1)
    _, M, N = o.get_state(0)
    q = 0.1 * 1.0 / (4.0 * 1.0)
    assert np.isclose(M[2, 3], q, rtol=1e-14, atol=0) and np.isclose(M[2, 2], -q, rtol=1e-14, atol=0)
    assert np.isclose(N[3, 2], q, rtol=1e-14, atol=0) and np.isclose(N[2, 2], -q, rtol=1e-14, atol=0)
    o.step(1)
    e = o.get_state(0)[0]
    depth = e + hh
    assert abs(depth[2, 2]) <= 1e-14
    for (j, i) in ((2, 1), (2, 3), (1, 2), (3, 2)):
        assert np.isclose(depth[j, i], q, rtol=1e-12, atol=0)
    b = o.budget(0)
    assert b["clip"] <= 1e-15 and abs(b["volume"] - v0) <= 1e-12 * v0


def test_velocity_limit_on_a_puddle(oracle_mod):
    """R12, the optional velocity limit: an interior face's flux is held to
    |flux| <= vel_limit x its face depth after the outflow limit. On the draining puddle of
    the outflow-limit pin the four front faces have the front depth D_f = eta_wet + h_dry
    = 0.1 m; with vel_limit = 0.1 m/s each carries exactly 0.1 x 0.1 = 0.01 m^2/s out
    (below the outflow limit's 0.025), so after the second mass update the puddle holds
    0.1 - 4 x 0.01 = 0.06 m and each neighbour 0.01 m; with the limit off the outflow
    limit decides, as in that pin. Volume is conserved and nothing is clipped."""
    nx = ny = 5
    blk, hh, nn = single(nx, ny, 1.0, -1.0)
    eta = np.full((ny, nx), 1.0)
    eta[2, 2] = 1.1
    for vlim, q in ((0.1, 0.01), (0.0, 0.025)):
        o = oracle_mod.Oracle([blk], [hh], [nn], dt=1.0, vel_limit=vlim)
        o.set_state(0, eta=eta)
        v0 = o.budget(0)["volume"]
        o.step(1)
        _, M, N = o.get_state(0)
        for got, sign in ((M[2, 3], 1), (M[2, 2], -1), (N[3, 2], 1), (N[2, 2], -1)):
            assert np.isclose(got, sign * q, rtol=1e-14, atol=0), (vlim, got)
        o.step(1)
        depth = o.get_state(0)[0] + hh
        assert np.isclose(depth[2, 2], 0.1 - 4 * q, rtol=1e-12, atol=1e-15)
        for (j, i) in ((2, 1), (2, 3), (1, 2), (3, 2)):
            assert np.isclose(depth[j, i], q, rtol=1e-12, atol=0)
        b = o.budget(0)
        assert b["clip"] <= 1e-15 and abs(b["volume"] - v0) <= 1e-12 * v0


def test_velocity_limit_leaves_open_water_alone_and_closes_the_budget(oracle_mod):
    """A 20 m/s limit never binds in open water (a 3 m wave on a 50 m shelf moves at about
    1 m/s): the open-water run with the limit on equals the run without it, bitwise;
    with a limit of 0.5 m/s it binds at the beach and the nested budget still closes."""
    from paper_2408_07609_gb300 import scenarios as S

    sc = S.coastal_hierarchy("vl", 5, (60, 54, 810.0), [(1, 36, 36), (1, 27, 27)], dt=0.5,
                             steps=0, shelf_w=8e3, slope_w=10e3, wiggle=1e3, coast_frac=0.6,
                             land_frac=0.4, source=dict(kind="gauss", sigma=4e3, peak=2.0))
    blk, hh, nn = single(40, 30, 500.0, 50.0, n=0.025, bc=(0, 0, 0, 0))
    x = centres(40, 500.0)
    y = centres(30, 500.0)
    bump = 3.0 * np.exp(-((x[None, :] - 10e3) ** 2 + (y[:, None] - 7e3) ** 2) / (2 * 2e3 ** 2))
    runs = []
    for vlim in (0.0, 20.0):
        o = oracle_mod.Oracle([blk], [hh], [nn], dt=5.0, vel_limit=vlim)
        o.set_initial_uplift(0, bump)
        o.step(200)
        runs.append(o.get_state(0))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    o = oracle_mod.Oracle(sc.blocks, sc.bathy, sc.manning, sc.dt, vel_limit=0.5)
    r = oracle_mod.Oracle(sc.blocks, sc.bathy, sc.manning, sc.dt)
    for oo in (o, r):
        for k, dz in enumerate(sc.uplift):
            if dz is not None:
                oo.set_initial_uplift(k, dz)
    v0 = [o.budget(k)["volume"] for k in range(3)]
    o.step(1500)
    r.step(1500)
    for k in range(3):
        b = o.budget(k)
        assert abs(b["volume"] - (v0[k] - b["outflow"] + b["clip"] + b["ring"])) <= 1e-12 * v0[k]
    assert any(not np.array_equal(o.get_state(k)[1], r.get_state(k)[1]) for k in range(3))


def test_full_feedback_exchange_is_simultaneous(oracle_mod):
    """Full feedback with three levels: every level's means are formed before any level
    receives, as in a pack-then-unpack exchange. So one step of the three-level nest
    leaves the root exactly where the same step of the nest without the grandchild
    leaves it (the root sees the child's own levels), while the grandchild, whose levels
    differ from the child's, does change the child."""
    dxp, h = 300.0, 10.0
    P = dict(level=1, parent=-1, nx=90, ny=30, i0=0, j0=0, dx=dxp, bc=(1, 1, 0, 0))
    Cb = dict(level=2, parent=0, nx=90, ny=54, i0=30, j0=6, dx=dxp / 3, bc=(0,) * 4)
    G = dict(level=3, parent=1, nx=45, ny=36, i0=30, j0=20, dx=dxp / 9, bc=(0,) * 4)

    def arrays(b):
        return np.full((b["ny"], b["nx"]), h), np.zeros((b["ny"], b["nx"]), np.float32)

    def pulse(b, x0, y0, amp, cx, cy):
        x, y = np.meshgrid(x0 + centres(b["nx"], b["dx"]), y0 + centres(b["ny"], b["dx"]))
        return amp * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * 2000.0 ** 2))

    cx, cy = 45 * dxp, 15 * dxp
    eP = pulse(P, 0.0, 0.0, 0.1, cx, cy)
    eC = pulse(Cb, 30 * dxp, 6 * dxp, 0.1, cx, cy)
    eG = pulse(G, 30 * dxp + 30 * dxp / 3, 6 * dxp + 20 * dxp / 3, 0.3, cx, cy)  # not the child's
    runs = {}
    for name, bl in (("three", [P, Cb, G]), ("two", [P, Cb])):
        hs, ns = zip(*[arrays(b) for b in bl])
        o = oracle_mod.Oracle(bl, list(hs), list(ns), dt=1.0, nest_feedback=oracle_mod.NEST_FULL)
        o.set_state(0, eta=eP)
        o.set_state(1, eta=eC)
        if len(bl) == 3:
            o.set_state(2, eta=eG)
        o.step(1)
        runs[name] = o
    for a, b in zip(runs["three"].get_state(0), runs["two"].get_state(0)):
        assert np.array_equal(a, b)
    c3, c2 = runs["three"].get_state(1)[0], runs["two"].get_state(1)[0]
    assert np.abs(c3 - c2).max() > 1e-3  # the grandchild's means reached the child


def test_initial_condition_r10(oracle_mod):
    """R10: eta0 = max(dz, -h) on sea cells and -h on land whatever dz is; fluxes zero;
    the maximum and the arrival start from eta0 (a cell at or above the threshold has
    arrived at t = 0, a dry cell has no maximum)."""
    nx, ny = 6, 4
    h = np.array([[5.0, 5.0, 1.0, 0.5, -1.0, -2.0]] * ny)
    blk, _, nn = single(nx, ny, 100.0, 0.0)
    o = oracle_mod.Oracle([blk], [h], [nn], dt=1.0)
    dz = np.array([[0.02, -7.0, -1.0, 0.005, 3.0, -0.5]] * ny)
    o.set_initial_uplift(0, dz)
    e, M, N = o.get_state(0)
    want = np.array([[0.02, -5.0, -1.0, 0.005, 1.0, 2.0]] * ny)
    assert np.array_equal(e, want)
    assert not M.any() and not N.any()
    mh, at = o.max_height(0), o.arrival_time(0)
    wet = h + want > 1e-3
    assert np.array_equal(np.isnan(mh), ~wet)
    assert np.array_equal(mh[wet], want[wet])
    assert np.array_equal(at, np.where(wet & (want >= 0.01), 0.0, -1.0))


def test_friction_takes_the_rougher_neighbour(oracle_mod):
    """R2 friction at a face between cells of different roughness uses n_f = max(nL, nR)
    (the stated reading). Uniform flow M0 over a flat bottom with Manning n alternating
    by column (x faces) and by row (y faces): away from the walls, one step gives
    M1 = (1 - F) M0 / (1 + F) with F = (dt/2) g n_f^2 |M0| / D^(7/3) on every face, and
    the face between a smooth and a rough cell decays like the rough one."""
    nx, ny, hd, dt, dx = 16, 16, 10.0, 1.0, 100.0
    n = np.where((np.arange(nx)[None, :] + np.arange(ny)[:, None]) % 2 == 0, 0.02, 0.05)
    blk, hh, _ = single(nx, ny, dx, hd)
    o = oracle_mod.Oracle([blk], [hh], [n.astype(np.float32)], dt=dt)
    M0 = 1.0
    M = np.full((ny, nx + 1), M0)
    M[:, 0] = M[:, nx] = 0.0
    Nf = np.full((ny + 1, nx), M0)
    Nf[0, :] = Nf[ny, :] = 0.0
    o.set_state(0, eta=np.zeros((ny, nx)), M=M, N=Nf)
    o.step(1)
    _, M1, N1 = o.get_state(0)
    n32 = n.astype(np.float32).astype(np.float64)
    for f in range(4, nx - 3):  # x faces clear of the walls' influence, rows clear too
        for j in range(4, ny - 4):
            nf = max(n32[j, f - 1], n32[j, f])
            F = 0.5 * dt * G * nf * nf * math.sqrt(M0 * M0 + M0 * M0) / (hd * hd * np.cbrt(hd))
            assert math.isclose(M1[j, f], (1 - F) * M0 / (1 + F), rel_tol=1e-13), (j, f)
    for g in range(4, ny - 3):
        for i in range(4, nx - 4):
            nf = max(n32[g - 1, i], n32[g, i])
            F = 0.5 * dt * G * nf * nf * math.sqrt(M0 * M0 + M0 * M0) / (hd * hd * np.cbrt(hd))
            assert math.isclose(N1[g, i], (1 - F) * M0 / (1 + F), rel_tol=1e-13), (g, i)


def test_dry_basin_with_open_edges_stays_dry(oracle_mod):
    """R6 radiation needs a wet edge cell: an empty basin (every sea cell dry, eta = -h,
    ground below sea level) with radiation on all four edges has no water to move, so
    it stays empty, bitwise, with nothing crossing its edges."""
    nx, ny = 12, 10
    rng = np.random.default_rng(3)
    h = rng.uniform(0.5, 8.0, (ny, nx))
    h[3:5, 6:9] = -2.0  # some land too
    blk, _, nn = single(nx, ny, 100.0, 0.0, n=0.03, bc=(1, 1, 1, 1))
    o = oracle_mod.Oracle([blk], [h], [nn], dt=1.0)
    o.set_state(0, eta=-h)
    o.step(100)
    e, M, N = o.get_state(0)
    assert np.array_equal(e, -h)
    assert not M.any() and not N.any()
    assert o.budget(0)["outflow"] == 0.0
