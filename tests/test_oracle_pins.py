"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an exact identity, an invariance, a scaling law the paper states, a
Monte-Carlo brute force of the electrons a macro-particle stands for, or a
quadrature of the Table 1 shapes.  All run on the CPU.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle

C = 299792458.0


def circular_orbit(beta, rho, t):
    """Circular orbit of radius rho in the x-y plane, speed beta c (arrays for one particle)."""
    w0 = beta * C / rho
    ps = w0 * t
    r = np.array([rho * math.cos(ps), rho * math.sin(ps), 0.0])
    b = np.array([-beta * math.sin(ps), beta * math.cos(ps), 0.0])
    bd = np.array([-beta * w0 * math.cos(ps), -beta * w0 * math.sin(ps), 0.0])
    return r, b, bd


def run_single(traj, bin_omega, bin_dir, times, dts, w=1.0, ff=(oracle.FF_POINT, 0.0)):
    acc = oracle.Accumulator(bin_omega, bin_dir, *ff)
    for t, dt in zip(times, dts):
        r, b, bd = traj(t)
        acc.accumulate(r, b, bd, np.array([w]), t, dt)
    return acc


# ---------------------------------------------------------------- Eq. 1
def test_circular_orbit_harmonics_closed_form():
    """Eq. 1 with K0, A and the phase: a circular orbit at harmonic m of
    w0 = beta c / rho, observed at angle Theta from the orbit normal, gives over
    N_p periods |int A chi dt|^2 = w^2 N_p^2 (2 pi/w0)^2 [cot^2 Th J_m(x)^2 +
    beta^2 J_m'(x)^2], x = m beta sin Th (Jacobi-Anger on the integration-by-parts
    form of Eq. 1)."""
    beta, rho = 0.6, 1e-6
    w0 = beta * C / rho
    period = 2 * math.pi / w0
    m_list, th_list = [1, 2, 5], [0.3, 1.0, math.pi / 2]
    bins = [(m, th) for m in m_list for th in th_list]
    bin_omega = np.array([m * w0 for m, _ in bins])
    bin_dir = np.array([[math.sin(th), 0.0, math.cos(th)] for _, th in bins])
    M, Np = 1200, 2
    dt = period / M
    times = np.arange(M * Np) * dt
    acc = run_single(lambda t: circular_orbit(beta, rho, t), bin_omega, bin_dir, times,
                     [dt] * len(times))
    got = acc.spectra()["tot"] / oracle.k0()
    for (m, th), g in zip(bins, got):
        x = m * beta * math.sin(th)
        jm = special.jv(m, x)
        jmp = 0.5 * (special.jv(m - 1, x) - special.jv(m + 1, x))
        want = (m * w0) ** 2 * Np**2 * period**2 * ((math.cos(th) / math.sin(th)) ** 2 * jm**2
                                                   + beta**2 * jmp**2)
        assert g == pytest.approx(want, rel=1e-9, abs=0), (m, th)


def test_amplitude_integration_by_parts_identity():
    """A = d/dt [n x (n x beta) / (1 - beta.n)], so int A e^{i phi} dt equals the
    boundary term minus i w int n x (n x beta) e^{i phi} dt with
    phi = w (t - n.r/c).  Checked on a non-periodic trajectory with trapezoid
    weights on both sides; this pins the amplitude formula and the phase sign."""
    gamma0, rho = 20.0, 2e-6
    bperp = 0.5 / gamma0
    wh = bperp * C / rho
    acc_z = 3e12  # longitudinal acceleration of beta_z, 1/s (keeps |beta| < 1 on the window)

    def traj(t):
        bz = 0.99 + acc_z * t
        r = np.array([rho * math.cos(wh * t), rho * math.sin(wh * t), C * (0.99 * t + 0.5 * acc_z * t * t)])
        b = np.array([-bperp * math.sin(wh * t), bperp * math.cos(wh * t), bz])
        bd = np.array([-bperp * wh * math.cos(wh * t), -bperp * wh * math.sin(wh * t), acc_z])
        return r, b, bd

    n_list = [np.array([math.sin(a), 0.0, math.cos(a)]) for a in (0.0, 0.02, 0.3)]
    om_list = [2e15, 7e15]
    bin_omega = np.array([o for _ in n_list for o in om_list])
    bin_dir = np.array([n for n in n_list for _ in om_list])
    T, K = 3e-15, 6000
    times = np.linspace(0.0, T, K + 1)
    h = times[1] - times[0]
    dts = np.full(K + 1, h)
    dts[0] = dts[-1] = h / 2
    acc = run_single(traj, bin_omega, bin_dir, times, dts)
    U = acc.amplitudes()["U"]
    for b, (om, n) in enumerate(zip(bin_omega, bin_dir)):
        def g(t):
            r, be, _ = traj(t)
            v = np.cross(n, np.cross(n, be))
            return v, 1.0 - be @ n, om * (t - n @ r / C)

        v0, d0, p0 = g(times[0])
        v1, d1, p1 = g(times[-1])
        boundary = v1 / d1 * np.exp(1j * p1) - v0 / d0 * np.exp(1j * p0)
        integ = np.zeros(3, complex)
        for t, dt in zip(times, dts):
            v, _, p = g(t)
            integ += dt * v * np.exp(1j * p)
        want = boundary - 1j * om * integ
        assert np.linalg.norm(U[b] - want) <= 2e-5 * np.linalg.norm(want), b


def test_amplitude_transverse_and_zero_without_acceleration():
    """n . A = 0 for any beta, beta_dot; beta_dot = 0 gives A = 0 and U = V = P = 0."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        b = rng.normal(size=3)
        b *= rng.uniform(0.1, 0.999) / np.linalg.norm(b)
        bd = rng.normal(size=3) * 1e14
        A = oracle.amplitude(n, b, bd)
        assert abs(A @ n) <= 1e-13 * np.linalg.norm(A)
    n = np.array([0.0, 0.0, 1.0])
    acc = oracle.Accumulator([1e15, 3e16], [n, n])
    r = rng.normal(size=(3, 5)) * 1e-6
    b = np.tile(np.array([[0.1], [0.0], [0.9]]), 5)
    acc.accumulate(r, b, np.zeros((3, 5)), np.full(5, 10.0), 1e-15, 1e-17)
    assert np.all(acc.acc == 0.0)


# ---------------------------------------------------------- invariances
def _random_bunch(rng, n):
    r = rng.normal(size=(3, n)) * 1e-6
    b = rng.normal(size=(3, n)) * 0.01
    b[2] = np.sqrt(1.0 - 1e-4 - b[0] ** 2 - b[1] ** 2)
    bd = rng.normal(size=(3, n)) * 1e13
    w = rng.uniform(1.0, 50.0, n)
    return r, b, bd, w


def test_time_shift_translation_rotation():
    """A common time shift T multiplies U, V, P by e^{i w T}; a translation d by
    e^{-i w n.d/c}; a rotation of trajectories and directions leaves the spectra
    unchanged (Eq. 1 depends on t - n.r/c and on dot/cross products only)."""
    rng = np.random.default_rng(3)
    r, b, bd, w = _random_bunch(rng, 7)
    dirs = np.array([[0.0, 0.0, 1.0], [0.01, 0.0, math.sqrt(1 - 1e-4)], [0.6, 0.0, 0.8]])
    om = np.array([1e15, 4e16])
    bo, bdir = oracle.grid_bins(om, dirs)
    ts = np.arange(20) * 1e-16

    def run(r_, b_, bd_, dirs_, t_off=0.0):
        bo_, bdir_ = oracle.grid_bins(om, dirs_)
        acc = oracle.Accumulator(bo_, bdir_, oracle.FF_GAUSS, 0.1e-6)
        for t in ts:
            acc.accumulate(r_, b_, bd_, w, t + t_off, 1e-16)
        return acc

    base = run(r, b, bd, dirs)
    U0 = base.amplitudes()
    T = 3.3e-13
    sh = run(r, b, bd, dirs, t_off=T).amplitudes()
    for k in ("U", "V", "P"):
        np.testing.assert_allclose(sh[k], U0[k] * np.exp(1j * bo * T)[:, None], rtol=1e-8,
                                   atol=1e-8 * np.abs(U0[k]).max())
    d = np.array([2e-6, -1e-6, 5e-6])
    tr = run(r + d[:, None], b, bd, dirs).amplitudes()
    ph = np.exp(-1j * bo * (bdir @ d) / C)
    np.testing.assert_allclose(tr["U"], U0["U"] * ph[:, None], rtol=1e-9,
                               atol=1e-9 * np.abs(U0["U"]).max())
    # random rotation
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    rot = run(q @ r, q @ b, q @ bd, dirs @ q.T)
    s0, s1 = base.spectra(), rot.spectra()
    for k in ("coh", "inc", "tot", "paper"):
        np.testing.assert_allclose(s1[k], s0[k], rtol=1e-9)


# ------------------------------------------------------------- scaling
def _short_helix(n_steps=40):
    gamma, rho = 30.0, 1e-6
    bperp = 1.0 / gamma
    wh = bperp * C / rho
    bz = math.sqrt(1 - 1 / gamma**2 - bperp**2)

    def traj(t, phase=0.0):
        p = wh * t + phase
        r = np.array([rho * math.cos(p), rho * math.sin(p), bz * C * t])
        b = np.array([-bperp * math.sin(p), bperp * math.cos(p), bz])
        bd = np.array([-bperp * wh * math.cos(p), -bperp * wh * math.sin(p), 0.0])
        return r, b, bd

    return traj, np.arange(n_steps) * 2e-17, 2e-17


def test_coherent_scaling_n_squared():
    """N identical co-located point electrons radiate N^2 times one (Sec. 3.2, point
    charge fully coherent); so does one point macro-particle of weight N."""
    traj, times, dt = _short_helix()
    bo, bdir = oracle.grid_bins([1e15, 1e16, 1e17], [[0, 0, 1.0], [0.02, 0, math.sqrt(1 - 4e-4)]])
    N = 9
    one = oracle.Accumulator(bo, bdir)
    many = oracle.Accumulator(bo, bdir)
    macro = oracle.Accumulator(bo, bdir)
    for t in times:
        r, b, bd = traj(t)
        one.accumulate(r, b, bd, [1.0], t, dt)
        many.accumulate(np.repeat(r[:, None], N, 1), np.repeat(b[:, None], N, 1),
                        np.repeat(bd[:, None], N, 1), np.ones(N), t, dt)
        macro.accumulate(r, b, bd, [float(N)], t, dt)
    i1 = one.spectra()["tot"]
    np.testing.assert_allclose(many.spectra()["tot"], N**2 * i1, rtol=1e-12)
    sm = macro.spectra()
    np.testing.assert_allclose(sm["tot"], N**2 * i1, rtol=1e-12)
    np.testing.assert_allclose(sm["coh"], N**2 * i1, rtol=1e-12)
    assert np.all(sm["inc"] == 0.0)


def test_incoherent_scaling_n():
    """N electrons at random offsets along n spread over L >> c/omega radiate on
    average N times one electron (random relative phases)."""
    traj, times, dt = _short_helix(n_steps=16)
    om = 2e17
    n = np.array([0.0, 0.0, 1.0])
    one = oracle.Accumulator([om], [n])
    for t in times:
        r, b, bd = traj(t)
        one.accumulate(r, b, bd, [1.0], t, dt)
    i1 = one.spectra()["tot"][0]
    N, seeds = 12, 150
    vals = []
    for s in range(seeds):
        rng = np.random.default_rng(100 + s)
        off = rng.uniform(0.0, 50e-6, N)  # >> c / omega = 1.5 nm
        acc = oracle.Accumulator([om], [n])
        for t in times:
            r, b, bd = traj(t)
            rr = np.repeat(r[:, None], N, 1)
            rr[2] += off
            acc.accumulate(rr, np.repeat(b[:, None], N, 1), np.repeat(bd[:, None], N, 1),
                           np.ones(N), t, dt)
        vals.append(acc.spectra()["tot"][0])
    vals = np.array(vals)
    mean, se = vals.mean(), vals.std(ddof=1) / math.sqrt(seeds)
    assert abs(mean - N * i1) <= 5 * se, (mean / i1, se / i1)


# -------------------------------------------------------- form factors
def _shape_density(name, x, width):
    """rho(x) of Table 1: box of width Delta convolved p-1 times (cardinal B-splines),
    or the normalised Gaussian; each integrates to one."""
    a = np.abs(x) / width
    if name == "CIC":
        return np.where(a <= 0.5, 1.0, 0.0) / width
    if name == "TSC":
        return np.where(a <= 1.0, 1.0 - a, 0.0) / width
    if name == "QSC":
        return np.where(a <= 0.5, 0.75 - a * a, np.where(a <= 1.5, 0.5 * (1.5 - a) ** 2, 0.0)) / width
    if name == "Gauss":
        return np.exp(-0.5 * (x / width) ** 2) / (math.sqrt(2 * math.pi) * width)
    raise ValueError(name)


def _read_table1():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_form_factors.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, p, sinc_pow, gexp = line.split()
                rows.append((name, int(p), int(sinc_pow), int(gexp)))
    return rows


KIND = {"CIC": oracle.FF_CIC, "TSC": oracle.FF_TSC, "QSC": oracle.FF_QSC, "Gauss": oracle.FF_GAUSS}


def test_table1_by_quadrature():
    """f(omega) = int rho(x) e^{i omega x / c} dx for each Table 1 shape (fixture),
    by adaptive quadrature of the density, against the oracle's closed forms; also
    F^2 = f^2 has the printed sinc power / Gaussian exponent."""
    width = 0.1e-6
    for name, p, sinc_pow, gexp in _read_table1():
        support = {"CIC": 0.5, "TSC": 1.0, "QSC": 1.5, "Gauss": 12.0}[name] * width
        norm = integrate.quad(lambda x: _shape_density(name, x, width), -support, support,
                              limit=200, points=[-width / 2, 0.0, width / 2])[0]
        assert norm == pytest.approx(1.0, rel=1e-10, abs=0)
        for om in [0.0, 1e14, 3e15, 1e16, 4.7e16]:
            k = om / C
            want = integrate.quad(lambda x: _shape_density(name, x, width) * math.cos(k * x),
                                  -support, support, limit=400,
                                  points=[-width, -width / 2, 0.0, width / 2, width])[0]
            got = oracle.form_factor(KIND[name], width, om)[0]
            assert got == pytest.approx(want, rel=1e-8, abs=1e-12), (name, om)
            x = om * width / (2 * C)
            s = 1.0 if x == 0 else math.sin(x) / x
            F2 = s ** sinc_pow if gexp == 0 else math.exp(-gexp * (om * width / C) ** 2)
            assert got**2 == pytest.approx(F2, rel=1e-12, abs=1e-300)


def test_form_factor_limits():
    """f -> 1 (point shape, or omega -> 0) gives pure coherent w^2 |a|^2; f -> 0
    (Gaussian with omega sigma / c >> 1, CIC at sinc zeros) gives pure incoherent
    w |a|^2 (Sec. 3.2: continuous shapes kill high-frequency coherent emission;
    Eq. 12: N remains)."""
    traj, times, dt = _short_helix()
    w = 250.0
    n = [0.0, 0.0, 1.0]
    sig = 0.1e-6
    om_gauss = 41 * C / sig          # f^2 = e^{-1681}
    delta = 0.2e-6
    om_cic = 2 * math.pi * C / delta  # omega Delta / 2c = pi: a zero of the CIC sinc
    bo = np.array([1e12, om_gauss, om_cic])
    res = {}
    for name, ff in (("point", (oracle.FF_POINT, 0.0)), ("gauss", (oracle.FF_GAUSS, sig)),
                     ("cic", (oracle.FF_CIC, delta)), ("one", (oracle.FF_POINT, 0.0))):
        acc = oracle.Accumulator(bo, [n] * 3, *ff)
        for t in times:
            r, b, bd = traj(t)
            acc.accumulate(r, b, bd, [1.0 if name == "one" else w], t, dt)
        res[name] = acc.spectra()
    a2 = res["one"]["tot"]
    np.testing.assert_allclose(res["point"]["tot"], w**2 * a2, rtol=1e-12)
    assert np.all(res["point"]["inc"] == 0)
    assert res["gauss"]["coh"][1] == 0.0
    assert res["gauss"]["tot"][1] == pytest.approx(w * a2[1], rel=1e-12, abs=0)
    assert res["gauss"]["tot"][0] == pytest.approx(w**2 * a2[0], rel=1e-6, abs=0)  # omega sigma/c = 3e-4
    assert res["cic"]["coh"][2] <= 1e-28 * w**2 * a2[2]
    assert res["cic"]["tot"][2] == pytest.approx(w * a2[2], rel=1e-12, abs=0)


def test_split_equals_literal_for_uniform_weights_and_single_particle():
    """The paper's literal in-situ sum |sum F_k A chi|^2 (Eq. 13) equals the split
    readout I_coh + I_inc when all weights are equal, and for one macro-particle."""
    rng = np.random.default_rng(11)
    r, b, bd, _ = _random_bunch(rng, 6)
    bo, bdir = oracle.grid_bins([1e14, 2e15, 3e16], [[0, 0, 1.0], [0.3, 0, math.sqrt(0.91)]])
    for w, sl in ((np.full(6, 37.0), slice(None)), (np.array([123.0]), slice(0, 1))):
        acc = oracle.Accumulator(bo, bdir, oracle.FF_TSC, 0.3e-6)
        for t in np.arange(8) * 1e-16:
            acc.accumulate(r[:, sl], b[:, sl], bd[:, sl], w, t, 1e-16)
        s = acc.spectra()
        np.testing.assert_allclose(s["paper"], s["tot"], rtol=1e-12)


@pytest.mark.parametrize("shape", ["CIC", "TSC", "QSC", "Gauss"])
def test_brute_force_electrons_match_form_factor(shape):
    """Sec. 3.2 (Eq. 7-12): replace each macro-particle by w electrons at static
    offsets drawn from its shape, average |sum|^2 over realisations: the mean
    equals K0 [f^2 |sum w_k a_k|^2 + (1 - f^2) sum w_k |a_k|^2], i.e. the split
    coherent part plus the exact incoherent part; for one macro-particle it is
    the oracle's I_tot.  Pins Table 1's normalisation and sinc convention."""
    rng = np.random.default_rng({"CIC": 1, "TSC": 2, "QSC": 3, "Gauss": 4}[shape])
    traj, times, dt = _short_helix(n_steps=12)
    width = 0.1e-6
    n = np.array([0.0, 0.0, 1.0])
    x_half = {"CIC": 1.0, "TSC": 1.1, "QSC": 1.2, "Gauss": 0.9}[shape]
    om = x_half * 2 * C / width if shape != "Gauss" else x_half * C / width  # f^2 in (0.2, 0.8)
    w_list = [6, 4]
    centers = [np.zeros(3), np.array([0.0, 0.0, 0.37e-6])]
    R = 1500
    # macro-particle computation
    acc = oracle.Accumulator([om], [n], KIND[shape], width)
    a_parts = None
    for t in times:
        r, b, bd = traj(t)
        rr = np.stack([r + c for c in centers], axis=1)
        bb = np.repeat(b[:, None], 2, 1)
        dd = np.repeat(bd[:, None], 2, 1)
        acc.accumulate(rr, bb, dd, np.array(w_list, float), t, dt)
        a_parts = oracle.accumulate_particles([om], [n], rr, bb, dd, t, dt, a_parts)
    f2 = oracle.form_factor(KIND[shape], width, om)[0] ** 2
    a = oracle.complex_particles(a_parts)[:, 0, :]  # [2][3]
    k0 = oracle.k0()
    inc_exact = k0 * (1 - f2) * sum(wk * np.vdot(a[k], a[k]).real for k, wk in enumerate(w_list))
    want = acc.spectra()["coh"][0] + inc_exact

    # brute force: every electron a separate point particle at a drawn offset
    def draw(m):
        if shape == "Gauss":
            return rng.normal(0.0, width, size=(3, m))
        u = sum(rng.uniform(-0.5, 0.5, m) for _ in range({"CIC": 1, "TSC": 2, "QSC": 3}[shape]))
        return np.stack([np.zeros(m), np.zeros(m), u * width])  # offsets along n (Table 1 is 1D)

    ne = sum(w_list)
    offs = [draw(ne) for _ in range(R)]
    owner = np.repeat(np.arange(2), w_list)
    el = None
    for t in times:
        r, b, bd = traj(t)
        rr = np.concatenate([np.stack([r + centers[o] for o in owner], 1) + off for off in offs], 1)
        m = rr.shape[1]
        el = oracle.accumulate_particles([om], [n], rr, np.repeat(b[:, None], m, 1),
                                         np.repeat(bd[:, None], m, 1), t, dt, el)
    z = oracle.complex_particles(el)[:, 0, :].reshape(R, ne, 3).sum(axis=1)
    vals = k0 * np.sum(np.abs(z) ** 2, axis=1)
    mean, se = vals.mean(), vals.std(ddof=1) / math.sqrt(R)
    assert abs(mean - want) <= 5 * se, (mean / want, se / want)
    assert se / want < 0.05
    # single macro-particle: the split readout is the brute-force expectation
    one = oracle.Accumulator([om], [n], KIND[shape], width)
    for t in times:
        r, b, bd = traj(t)
        one.accumulate(r, b, bd, [6.0], t, dt)
    s1 = one.spectra()
    np.testing.assert_allclose(s1["paper"], s1["tot"], rtol=1e-12)


# ------------------------------------------------ absolute normalisation
def test_energy_integral_equals_lienard_power():
    """Integrating the oracle's spectrum over omega in [0, inf) and the full solid
    angle gives the total radiated energy (Eq. 1 is the energy per unit frequency
    and solid angle).  For a charge with a Gaussian acceleration pulse along its
    velocity this must equal the Lienard energy int q^2 gamma^6 betadot^2 /
    (6 pi eps0 c) dt.  Pins the absolute prefactor K0 independently of Eq. 1."""
    qe, eps0 = 1.602176634e-19, 8.8541878128e-12
    b0, db, tau = 0.15, 0.1, 1e-15
    M = 1601
    times = np.linspace(-8 * tau, 8 * tau, M)
    h = times[1] - times[0]
    x = times / tau
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)
    cdf = 0.5 * (1 + special.erf(x / math.sqrt(2)))
    beta = b0 + db * cdf
    z = C * (b0 * times + db * tau * (x * cdf + pdf))
    bdot = db * pdf / tau
    mu, wmu = np.polynomial.legendre.leggauss(48)
    om_nodes, w_om = np.polynomial.legendre.leggauss(80)
    om_max = 2.4e16
    om = 0.5 * om_max * (om_nodes + 1)
    w_om = 0.5 * om_max * w_om
    dirs = np.stack([np.sqrt(1 - mu * mu), np.zeros_like(mu), mu], axis=1)
    bo, bdir = oracle.grid_bins(om, dirs)
    acc = oracle.Accumulator(bo, bdir)
    for j, t in enumerate(times):
        acc.accumulate([0.0, 0.0, z[j]], [0.0, 0.0, beta[j]], [0.0, 0.0, bdot[j]], [1.0], t, h)
    spec = acc.spectra()["tot"].reshape(len(mu), len(om))
    energy = 2 * math.pi * np.einsum("i,ij,j->", wmu, spec, w_om)
    gamma = 1.0 / np.sqrt(1 - beta * beta)
    lienard = np.sum(qe**2 * gamma**6 * bdot**2 / (6 * math.pi * eps0 * C)) * h
    assert energy == pytest.approx(lienard, rel=1e-6, abs=0)


# ------------------------------------------- direction-dependent box shapes
def test_form_factor_3d_reduces_to_table1_along_axes():
    """The axis-aligned 3-D box product equals the 1-D Table 1 form along a
    coordinate axis (the other factors are sinc(0) = 1) and differs off-axis."""
    width = 0.2e-6
    for kind in (oracle.FF_CIC, oracle.FF_TSC, oracle.FF_QSC):
        for om in (3e14, 2e15, 9e15):
            f1 = oracle.form_factor(kind, width, om)[0]
            for axis in np.eye(3):
                assert oracle.form_factor_dir(kind, oracle.FF_3D, width, om, axis) == f1
            n = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
            f3 = oracle.form_factor_dir(kind, oracle.FF_3D, width, om, n)
            want = np.prod([oracle.form_factor(kind, width, om * c)[0] for c in n])
            assert f3 == pytest.approx(want, rel=1e-14, abs=0)
    # the isotropic Gaussian ignores the flag
    n = np.array([0.6, 0.0, 0.8])
    assert oracle.form_factor_dir(oracle.FF_GAUSS, oracle.FF_3D, 0.1e-6, 1e15, n) == \
        oracle.form_factor(oracle.FF_GAUSS, 0.1e-6, 1e15)[0]


@pytest.mark.parametrize("shape", ["CIC", "TSC"])
def test_brute_force_3d_box_offsets_oblique_direction(shape):
    """Electrons offset by an axis-aligned 3-D box distribution, seen along an
    oblique direction: the Monte-Carlo mean of |sum|^2 matches the 3-D product
    form factor (Sec. 3.2 with rho = rho(x) rho(y) rho(z)) and not the 1-D form."""
    rng = np.random.default_rng(21)
    traj, times, dt = _short_helix(n_steps=10)
    width = 0.15e-6
    n = np.array([0.5, -0.6, math.sqrt(1 - 0.25 - 0.36)])
    om = {"CIC": 3.0, "TSC": 2.0}[shape] * 2 * C / width  # omega Delta / 2c along a unit axis
    kind = KIND[shape]
    w = 12
    R = 1500
    macro = oracle.Accumulator([om], [n], kind, width, oracle.FF_3D)
    for t in times:
        r, b, bd = traj(t)
        macro.accumulate(r, b, bd, [float(w)], t, dt)
    want = macro.spectra()["tot"][0]
    want_1d = macro.spectra(ff_flags=0)["tot"][0]
    m = {"CIC": 1, "TSC": 2}[shape]
    offs = [sum(rng.uniform(-0.5, 0.5, (3, w)) for _ in range(m)) * width for _ in range(R)]
    el = None
    for t in times:
        r, b, bd = traj(t)
        rr = np.concatenate([r[:, None] + o for o in offs], 1)
        k = rr.shape[1]
        el = oracle.accumulate_particles([om], [n], rr, np.repeat(b[:, None], k, 1),
                                         np.repeat(bd[:, None], k, 1), t, dt, el)
    z = oracle.complex_particles(el)[:, 0, :].reshape(R, w, 3).sum(axis=1)
    vals = oracle.k0() * np.sum(np.abs(z) ** 2, axis=1)
    mean, se = vals.mean(), vals.std(ddof=1) / math.sqrt(R)
    assert abs(mean - want) <= 5 * se, (mean / want, se / want)
    assert abs(mean - want_1d) > 5 * se  # the direction dependence is resolved


def test_species_single_and_split_population():
    """One species reads out exactly as the single-shape readout.  A population
    split into two species of the same shape has the coherent part of one
    accumulator fed all particles (the species' amplitudes add before |.|^2,
    Eq. 13 with one f for all macro-particles), and an incoherent part that is
    the sum of the species' own incoherent parts (Eq. 12 per species: no
    cross-species terms)."""
    rng = np.random.default_rng(23)
    r, b, bd, w = _random_bunch(rng, 10)
    bo, bdir = oracle.grid_bins([2e14, 3e15, 5e16], [[0, 0, 1.0], [0.3, -0.2, math.sqrt(0.87)]])
    for ff in ((oracle.FF_TSC, 0.4e-6), (oracle.FF_CIC, 0.3e-6, oracle.FF_3D)):
        flags = ff[2] if len(ff) > 2 else 0
        whole = oracle.Accumulator(bo, bdir, ff[0], ff[1], flags)
        parts = [oracle.Accumulator(bo, bdir, ff[0], ff[1], flags) for _ in range(2)]
        for t in np.arange(6) * 1e-16:
            whole.accumulate(r, b, bd, w, t, 1e-16)
            for acc, sl in zip(parts, (slice(0, 4), slice(4, 10))):
                acc.accumulate(r[:, sl], b[:, sl], bd[:, sl], w[sl], t, 1e-16)
        want = whole.spectra()
        one = oracle.species_spectra([whole], [ff])
        two = oracle.species_spectra(parts, [ff, ff])
        for k in ("coh", "inc", "tot"):
            np.testing.assert_allclose(one[k], want[k], rtol=1e-13, atol=0)
        np.testing.assert_allclose(two["coh"], want["coh"], rtol=1e-12, atol=1e-300)
        inc_sum = parts[0].spectra()["inc"] + parts[1].spectra()["inc"]
        np.testing.assert_allclose(two["inc"], inc_sum, rtol=1e-12, atol=0)
        np.testing.assert_allclose(two["tot"], two["coh"] + two["inc"], rtol=1e-15, atol=0)
        assert np.all(want["inc"] > 0) and np.any(want["coh"] > 0)


def test_brute_force_two_species_of_different_shapes():
    """Sec. 3.2 per particle class: two macro-particles of different shapes (a
    CIC species and a Gaussian species) replaced by w electrons at offsets drawn
    from each one's own shape.  The mean of |sum|^2 over realisations equals
    K0 [|f_A w_A a_A + f_B w_B a_B|^2 + sum_s (1 - f_s^2) w_s |a_s|^2]: the
    species readout, whose coherent cross term carries f_A f_B."""
    rng = np.random.default_rng(29)
    traj, times, dt = _short_helix(n_steps=12)
    n = np.array([0.0, 0.0, 1.0])
    delta, sigma = 0.12e-6, 0.08e-6
    om = 1.0 * 2 * C / delta   # CIC: f^2 = sinc^2(1) ~ 0.71
    ffs = [(oracle.FF_CIC, delta), (oracle.FF_GAUSS, sigma)]
    f = [oracle.form_factor(k, wd, om)[0] for k, wd in ffs]
    assert 0.1 < f[0] ** 2 < 0.9 and 0.1 < f[1] ** 2 < 0.9
    w_list = [5, 7]
    centers = [np.zeros(3), np.array([0.0, 0.0, 0.29e-6])]
    accs = [oracle.Accumulator([om], [n], k, wd) for k, wd in ffs]
    for t in times:
        r, b, bd = traj(t)
        for s in range(2):
            accs[s].accumulate((r + centers[s])[:, None], b[:, None], bd[:, None],
                               np.array([float(w_list[s])]), t, dt)
    want = oracle.species_spectra(accs, ffs)["tot"][0]
    R = 1500

    def draw(s, m):
        if s == 1:
            return rng.normal(0.0, sigma, size=(3, m))
        return np.stack([np.zeros(m), np.zeros(m), rng.uniform(-0.5, 0.5, m) * delta])

    owner = np.repeat(np.arange(2), w_list)
    ne = owner.size
    offs = [np.concatenate([draw(s, w_list[s]) for s in range(2)], axis=1) for _ in range(R)]
    el = None
    for t in times:
        r, b, bd = traj(t)
        rr = np.concatenate([np.stack([r + centers[o] for o in owner], 1) + off for off in offs], 1)
        m = rr.shape[1]
        el = oracle.accumulate_particles([om], [n], rr, np.repeat(b[:, None], m, 1),
                                         np.repeat(bd[:, None], m, 1), t, dt, el)
    z = oracle.complex_particles(el)[:, 0, :].reshape(R, ne, 3).sum(axis=1)
    vals = oracle.k0() * np.sum(np.abs(z) ** 2, axis=1)
    mean, se = vals.mean(), vals.std(ddof=1) / math.sqrt(R)
    assert abs(mean - want) <= 5 * se, (mean / want, se / want)
    # the pin discriminates: reading both species with one shape, or dropping the
    # coherent cross term between species, misses by many sigma
    wrong = [oracle.species_spectra(accs, [ff, ff])["tot"][0] for ff in ffs]
    wrong.append(sum(a.spectra()["tot"][0] for a in accs))
    assert all(abs(mean - x) > 5 * se for x in wrong), [(x / want) for x in wrong]
