"""Pins for the FP64 forward-model oracle against closed forms, invariants and
independent formulations (no GPU).  Each test names what fixes the expected
value; none of them re-types the oracle's own formula.
"""
import numpy as np
import pytest
from scipy.special import erf

import oracle as O
from paper_2109_00661_gb300 import inputs as I

MU0 = 4e-7 * np.pi
A = 13.0


def h_total_halfspace(w, sig, a=A):
    """Ward & Hohmann (1988) closed form: total Hz at the centre of a loop of
    radius a on the surface of a uniform half-space (unit current)."""
    k = np.sqrt(-1j * w * MU0 * sig)
    k = np.where(np.imag(k) > 0, -k, k)
    return -(1.0 / (k ** 2 * a ** 3)) * (3 - (3 + 3j * k * a - k ** 2 * a ** 2) * np.exp(-1j * k * a))


def dhdt_step_off(t, sig, a=A):
    """Ward & Hohmann (1988) closed form: d hz/dt after a step-off, same geometry."""
    z = np.sqrt(MU0 * sig / (4 * t)) * a
    return -(1.0 / (MU0 * sig * a ** 3)) * (3 * erf(z) - (2 / np.sqrt(np.pi)) * z * (3 + 2 * z * z) * np.exp(-z * z))


# --------------------------------------------------------------------- Cole-Cole
def test_colecole_limits_and_m0():
    sig, m, tau, c = 0.05, 0.4, 1e-3, 0.6
    # m = 0 reduces to the conductive model (Section 2)
    assert O.colecole(0, sig, 0.0, tau, c, 123.0) == complex(sig, 0.0)
    # DC limit sigma_inf (1 - m), high-frequency limit sigma_inf
    lo = O.colecole(0, sig, m, tau, c, 1e-12)
    hi = O.colecole(0, sig, m, tau, c, 1e15)
    assert abs(lo - sig * (1 - m)) < 1e-6 * sig
    assert abs(hi - sig) < 1e-3 * sig
    # the conductivity is dispersive and causal: Im sigma > 0 in between
    assert O.colecole(0, sig, m, tau, c, 1.0 / tau).imag > 0


def test_colecole_paper_pelton_bijection():
    """Section 2 says the paper's form and Pelton's are related bijectively:
    sigma_inf = s0 / (1 - m) and tau^c = (1 - m) tau_p^c."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        s0 = 10 ** rng.uniform(-4, 0)
        m = rng.uniform(0.01, 0.95)
        taup = 10 ** rng.uniform(-6, -1)
        c = rng.uniform(0.1, 1.0)
        w = 10 ** rng.uniform(0, 8)
        pel = O.colecole(1, s0, m, taup, c, w)
        tau = taup * (1 - m) ** (1.0 / c)
        pap = O.colecole(0, s0 / (1 - m), m, tau, c, w)
        assert abs(pel - pap) <= 1e-12 * abs(pel)


def test_colecole_literal_form():
    """Pelton's expression taken as a conductivity (form 2): sigma_0 at DC and
    sigma_0 (1 - m) at high frequency, the paper's form with sigma_inf =
    sigma_0 (1 - m) and chargeability -m / (1 - m), and the product with
    Pelton's form (the reciprocal of the same expression times sigma_0^2)
    equal to sigma_0^2."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        s0 = 10 ** rng.uniform(-4, 0)
        m = rng.uniform(0.01, 0.95)
        tau = 10 ** rng.uniform(-6, -1)
        c = rng.uniform(0.1, 1.0)
        w = 10 ** rng.uniform(0, 8)
        lit = O.colecole(2, s0, m, tau, c, w)
        pap = O.colecole(0, s0 * (1 - m), -m / (1 - m), tau, c, w)
        assert abs(lit - pap) <= 1e-12 * abs(lit)
        assert abs(lit * O.colecole(1, s0, m, tau, c, w) - s0 * s0) <= 1e-12 * s0 * s0
        assert lit.real > 0 and lit.imag < 0  # the conductivity falls with frequency
    s0, m, tau, c = 0.05, 0.4, 1e-3, 0.6
    assert abs(O.colecole(2, s0, m, tau, c, 1e-12) - s0) < 1e-6 * s0
    assert abs(O.colecole(2, s0, m, tau, c, 1e15) - s0 * (1 - m)) < 1e-3 * s0
    assert O.colecole(2, s0, 0.0, tau, c, 123.0) == complex(s0, 0.0)


# --------------------------------------------------------------- recursion forms
def test_reflection_matches_admittance_recursion():
    rng = np.random.default_rng(4)
    for _ in range(40):
        L = rng.integers(1, 8)
        sig = 10 ** rng.uniform(-4, 1, L) * np.exp(1j * rng.uniform(0, 0.6, L))
        th = 10 ** rng.uniform(0, 2.3, L - 1)
        lam = 10 ** rng.uniform(-5, 0)
        w = 10 ** rng.uniform(1, 7)
        a = O.r0(sig, th, lam, w, 0)
        b = O.r0(sig, th, lam, w, 1)
        assert abs(a - b) <= 1e-9 * max(abs(a), 1e-300)


def test_split_layer_and_uniform_stack_invariants():
    sig = np.array([0.02, 0.2, 0.005])
    th = np.array([25.0, 40.0])
    lam, w = 0.02, 3e4
    base = O.r0(sig, th, lam, w)
    split = O.r0(np.array([0.02, 0.2, 0.2, 0.005]), np.array([25.0, 15.0, 25.0]), lam, w)
    assert abs(base - split) <= 1e-13 * abs(base)
    hs = O.r0(np.array([0.03]), [], lam, w)
    uni = O.r0(np.full(5, 0.03), np.full(4, 10.0), lam, w)
    assert abs(hs - uni) <= 1e-13 * abs(hs)
    # a vanishing conductivity gives a vanishing reflection (free space)
    assert abs(O.r0(np.array([1e-14]), [], lam, w)) < 1e-10


# ------------------------------------------------------------------ Hankel parts
@pytest.mark.parametrize("sig", [1e-3, 0.01, 0.3])
def test_hz_quadrature_closed_form_halfspace(sig):
    """Hz (total = primary I/(2a) + secondary) over a half-space at h = 0."""
    for w in [10.0, 1e3, 1e5, 1e7]:
        hs = O.hz([sig], [], A, 0.0, w, rtol=1e-12)
        ref = h_total_halfspace(w, sig)
        assert abs(hs + 1.0 / (2 * A) - ref) <= 1e-8 * abs(ref)


def test_hankel_rule_matches_quadrature_at_height():
    rng = np.random.default_rng(5)
    for K in (120, 200):
        for _ in range(12):
            L = rng.integers(1, 6)
            sig = 10 ** rng.uniform(-4, 0, L) * np.exp(1j * rng.uniform(0, 0.4, L))
            th = 10 ** rng.uniform(0.3, 2.3, L - 1)
            w = 2 * np.pi * 10 ** rng.uniform(0, 7)
            q = O.hz(sig, th, A, 30.0, w)
            r = O.hz(sig, th, A, 30.0, w, mode=O.HANKEL_RULE, K=K)
            assert abs(r - q) <= 1e-8 * abs(q)


@pytest.mark.parametrize("name", list(I.CONFIGS))
def test_hankel_rule_on_the_workload_draws(name):
    """The K-point rule against the adaptive quadrature on the random-model
    workload's own draws (1..10 layers, m up to 1, c up to 1, tau over five
    decades, Cole-Cole paper form), the whole forward model: Im Hz at every
    frequency node within 1e-6 of |Im Hz|, and every gate within 1e-6 of
    max(|y|, eps_an).  (Measured on 3000 throughput-workload models: spectrum
    max 1.9e-7, gates max 5.1e-7, median 6e-15.)"""
    s = I.oracle_system(name)
    s["T"] = O.tmatrix(s["freqs"], s["times"])
    models = I.random_models(400, seed=21)
    yq, imq = O.forward(models, s, mode=O.QUAD_REFLECTION, want_imh=True)
    yr, imr = O.forward(models, s, mode=O.HANKEL_RULE, want_imh=True)
    es = np.abs(imr - imq) / np.abs(imq)
    eg = np.abs(yr - yq) / np.maximum(np.abs(yq), I.EPS_AN)
    print(f"\n{name}: rule vs quadrature, spectrum max {es.max():.2e} median {np.median(es):.2e}; "
          f"gates max {eg.max():.2e} p99 {np.quantile(eg, 0.99):.2e} median {np.median(eg):.2e}")
    assert es.max() <= 1e-6 and eg.max() <= 1e-6


def test_hankel_rule_near_the_branch_point():
    """Where the rule loses accuracy: a half-space with m -> 1 and c -> 1 has
    sigma(w) nearly imaginary at w tau << 1, which puts the branch point of
    u = sqrt(lambda^2 + i w mu0 sigma) next to the real lambda axis and spoils
    the trapezoid rule's exponential convergence.  The spectrum error stays
    below 1e-3 of |Im Hz| there, and is within 1e-6 once m <= 0.9."""
    s = I.oracle_system("forward-g30-f60-k200")
    rng = np.random.default_rng(3)
    P = 200
    for mlo, mhi, tol in ((0.95, 0.9999, 1e-3), (0.5, 0.9, 1e-6)):
        models = dict(nlayers=np.full(P, 1, np.int8), logsig=rng.uniform(-4, 0, (P, 1)), logh=np.zeros((P, 1)),
                      m=rng.uniform(mlo, mhi, (P, 1)), logtau=rng.uniform(-6, -1, (P, 1)),
                      c=rng.uniform(0.9, 1.0, (P, 1)))
        imq = O.forward(models, s, mode=O.QUAD_REFLECTION, want_imh=True)[1]
        imr = O.forward(models, s, mode=O.HANKEL_RULE, want_imh=True)[1]
        es = np.abs(imr - imq) / np.abs(imq)
        print(f"\nhalf-spaces m in [{mlo}, {mhi}], c in [0.9, 1]: spectrum max {es.max():.2e} p99 {np.quantile(es, 0.99):.2e}")
        assert es.max() <= tol


# ------------------------------------------------------------- time transform
@pytest.fixture(scope="module")
def dense_T():
    freqs = np.logspace(0, 7, 400)
    times = np.logspace(-5, -2, 16)
    return freqs, times, O.tmatrix(freqs, times)


@pytest.mark.parametrize("sig,tol", [(0.1, 2e-4), (0.01, 2e-3)])
def test_tmatrix_step_off_closed_form(dense_T, sig, tol):
    freqs, times, T = dense_T
    hs = h_total_halfspace(2 * np.pi * freqs, sig) - 1.0 / (2 * A)
    y = T @ hs.imag
    ref = -MU0 * dhdt_step_off(times, sig)
    assert np.all(ref > 0)  # -dB/dt is positive for a conductive earth
    assert np.max(np.abs(y - ref) / ref) < tol


def test_tmatrix_exact_sine_transform(dense_T):
    """Int_0^inf w sin(w t) / (1 + (w tau)^2) dw = (pi / (2 tau^2)) e^{-t/tau}."""
    freqs, times, T = dense_T
    tau = 1e-3
    w = 2 * np.pi * freqs
    y = T @ (w / (1 + (w * tau) ** 2))
    ref = -(2 * MU0 / np.pi) * (np.pi / (2 * tau ** 2)) * np.exp(-times / tau)
    sel = times < 5e-3
    assert np.max(np.abs(y[sel] - ref[sel]) / np.abs(ref[sel])) < 1e-3


def test_forward_late_time_law_at_height():
    """At late times the step-off response of a half-space falls as t^(-5/2)
    with the coefficient a^2 (mu0 sigma)^(3/2) / (20 sqrt(pi)); the loop height
    enters only through a first-order correction of size ~ 2h / delta, with
    delta = sqrt(t / (mu0 sigma)) the diffusion depth."""
    sig = 1e-3
    freqs = np.logspace(-2, 7, 300)
    times = np.array([2e-3, 4e-3, 1e-2])
    late = MU0 * A ** 2 * (MU0 * sig) ** 1.5 / (20 * np.sqrt(np.pi) * times ** 2.5)
    for h in (30.0, 1.0):
        system = dict(a=A, h=h, freqs=freqs, times=times, K=200, cc_form=0)
        models = dict(nlayers=np.array([1]), logsig=np.array([[np.log10(sig)]]), logh=np.zeros((1, 1)),
                      m=np.zeros((1, 1)), logtau=np.full((1, 1), -3.0), c=np.ones((1, 1)))
        ratio = O.forward(models, system, mode=O.HANKEL_RULE)[0] / late
        small = 2 * h / np.sqrt(times / (MU0 * sig))
        assert np.all(np.abs(ratio - 1) < 1.5 * small + 0.025)


def test_forward_quadrature_vs_rule_and_m0():
    rng = np.random.default_rng(6)
    P, LMAX = 6, 4
    nl = rng.integers(1, LMAX + 1, P)
    models = dict(nlayers=nl, logsig=rng.uniform(-3, 0, (P, LMAX)), logh=rng.uniform(0.5, 2, (P, LMAX)),
                  m=rng.uniform(0, 0.6, (P, LMAX)), logtau=rng.uniform(-5, -2, (P, LMAX)),
                  c=rng.uniform(0.2, 1, (P, LMAX)))
    system = dict(a=A, h=30.0, freqs=np.logspace(0, 7, 40), times=np.logspace(-5, -2, 20), K=120, cc_form=0)
    system["T"] = O.tmatrix(system["freqs"], system["times"])
    yq = O.forward(models, system, mode=O.QUAD_REFLECTION)
    yr = O.forward(models, system, mode=O.HANKEL_RULE)
    den = np.maximum(np.abs(yq), 1e-13)
    assert np.max(np.abs(yq - yr) / den) < 1e-6
    # m = 0 everywhere gives the conductive model regardless of tau, c
    m0 = dict(models, m=np.zeros((P, LMAX)))
    m0b = dict(m0, logtau=m0["logtau"] - 1.0, c=1 - 0.5 * m0["c"])
    assert np.array_equal(O.forward(m0, system, mode=O.HANKEL_RULE), O.forward(m0b, system, mode=O.HANKEL_RULE))


def test_ip_layer_can_turn_late_gates_negative():
    """Fig. 1: a strongly chargeable second layer drives late-time values negative."""
    system = dict(a=A, h=30.0, freqs=np.logspace(0, 7, 60), times=np.logspace(-5, -2, 30), K=120, cc_form=0)
    base = dict(nlayers=np.array([3]), logsig=np.log10([[0.01, 0.1, 0.01]]), logh=np.log10([[20.0, 20.0, 1.0]]),
                logtau=np.full((1, 3), np.log10(4.07e-4)), c=np.ones((1, 3)))
    y0 = O.forward(dict(base, m=np.array([[0.0, 0.0, 0.0]])), system, mode=O.HANKEL_RULE)[0]
    y8 = O.forward(dict(base, m=np.array([[0.0, 0.8, 0.0]])), system, mode=O.HANKEL_RULE)[0]
    assert np.all(y0 > 0)
    assert np.any(y8 < 0)


# ----------------------------------------------------------------- likelihood
def test_loglik_two_gate_hand_example():
    # y_model = (2, -1), y_obs = (3, -1.5), eps_an = (1, 0.5), eps_mn = 0.5
    # v = (1 + 1, 0.25 + 0.25) = (2, 0.5); r = (1, -0.5)
    # l = -0.5 [1/2 + 0.25/0.5 + ln(2 pi 2) + ln(2 pi 0.5)] = -0.5 [1 + ln(2 pi^2 * 2 ... )]
    ll = O.loglik(np.array([[2.0, -1.0]]), np.array([3.0, -1.5]), np.array([1.0, 0.5]), 0.5)[0]
    expect = -0.5 * (0.5 + 0.5 + np.log(4 * np.pi) + np.log(np.pi))
    assert abs(ll - expect) < 1e-14


def test_merge_direct_sum():
    # conductive interfaces at 10, 50 (sigma -2, -1, -3); IP interface at 30 (m 0.4)
    th, ls, m = O.merge([10.0, 50.0], [-2.0, -1.0, -3.0], [30.0], [0.4])
    assert np.allclose(th[:-1], [10.0, 20.0, 20.0])
    assert np.allclose(ls, [-2.0, -1.0, -1.0, -3.0])
    assert np.allclose(m, [0.0, 0.0, 0.4, 0.4])


def test_fd_gradient_is_step_consistent():
    """The oracle's central-difference gradient agrees between two step sizes
    (its truncation error is O(step^2): below 1e-5 of the gradient scale at the
    default step of 1e-5)."""
    from paper_2109_00661_gb300 import inputs as I
    rng = np.random.default_rng(8)
    P = 4
    models = dict(nlayers=np.full(P, 3), logsig=np.log10([[0.01, 0.1, 0.01]] * P) + rng.uniform(-0.2, 0.2, (P, 3)),
                  logh=np.log10([[20.0, 30.0, 1.0]] * P) + rng.uniform(-0.1, 0.1, (P, 3)),
                  m=rng.uniform(0.05, 0.5, (P, 3)), logtau=np.full((P, 3), -3.0) + rng.uniform(-0.3, 0.3, (P, 3)),
                  c=rng.uniform(0.3, 0.9, (P, 3)))
    s = I.oracle_system("sounding-g20-f40-k120")
    s["T"] = O.tmatrix(s["freqs"], s["times"])
    y_obs = I.noisy(O.forward(I.truth_3layer(), s, mode=O.HANKEL_RULE)[0], seed=0)
    _, g1 = O.loglik_grad_fd(models, s, y_obs, I.EPS_AN, I.EPS_MN, step=2e-5)
    _, g2 = O.loglik_grad_fd(models, s, y_obs, I.EPS_AN, I.EPS_MN, step=1e-5)
    scale = np.max(np.abs(g2), axis=(1, 2), keepdims=True)
    assert np.max(np.abs(g1 - g2) / scale) < 1e-5
    # the gate Jacobian reproduces it through the chain rule with the
    # closed-form d ll / d yhat (Section 2.3.2's Gaussian likelihood)
    from parity_util import dll_dy
    y, J = O.forward_jacobian_fd(models, s)
    g3 = np.einsum("pg,pgnk->pnk", dll_dy(y, y_obs), J)
    assert np.max(np.abs(g3 - g2) / scale) < 1e-6
