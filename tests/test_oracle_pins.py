"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a closed form, an exact identity,
brute force on a tiny input, an Euler-Maclaurin error term or a statistical
law, chosen so that a dropped term, a flipped sign, a shifted index or a
transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- spectrum --
def test_spectrum_matches_direct_dft():
    """Step 2 (Section 4): brute-force DFT sum on a tiny series."""
    rng = np.random.default_rng(3)
    n = 48
    x = rng.standard_normal(n)
    X = O.spectrum(x)
    assert X.shape == (n // 2,)
    for k in range(n // 2):
        ref = sum(x[t] * complex(math.cos(2 * math.pi * k * t / n),
                                 -math.sin(2 * math.pi * k * t / n)) for t in range(n))
        assert abs(X[k] - ref) < 1e-12 * n


# ------------------------------------------------------------- templates --
@pytest.mark.parametrize("n", [1 << 12, 1 << 14])
@pytest.mark.parametrize("z", [-50.0, -7.0, -2.0, 2.0, 36.0, 50.0])
def test_fresnel_template_vs_discrete_euler_maclaurin(n, z):
    """Section 2 template. The exact response of a sampled chirp is the
    left-endpoint sum (1/n) sum_k f(k/n) of the integrand f of the continuous
    template. Because f(1) = f(0) for integer d, Euler-Maclaurin gives
    discrete - continuous = (f'(1) - f'(0)) / (12 n^2) + O(n^-4)
                          = -i pi z / (6 n^2) + O(n^-4)."""
    m = 128
    tf = O.template_fresnel(z, m)
    td = O.template_discrete(z, m, n)
    pred = -1j * math.pi * z / (6.0 * n * n)
    resid = np.max(np.abs(td - tf - pred))
    bound = 2.0 * (2 * math.pi * (m / 2 + abs(z))) ** 3 / (720.0 * n ** 4)
    assert resid <= bound + 1e-14, (resid, bound)
    # the leading term itself is visible (the closed form is not accidentally
    # equal to the discrete sum for a wrong reason)
    assert np.max(np.abs(td - tf)) > 0.5 * abs(pred)


@pytest.mark.parametrize("z", [-6.0, 0.0, 4.0, 5.0])
def test_full_width_discrete_template_equals_brute_force_chirped_dft(z):
    """With all n taps of the discrete template, the correlation
    sum_d X[r+d] tau_z(d) (circular over the complex spectrum) equals the
    brute-force chirped DFT sum_n x_n exp(-2 pi i ((r - z/2) n/n + z n^2/(2 n^2)))
    exactly; r labels the chirp's mean frequency."""
    n = 64
    rng = np.random.default_rng(0)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = np.fft.fft(x)
    tau = O.template_discrete(z, n, n)
    d = np.arange(-n // 2, n // 2)
    t = np.arange(n)
    for r in (0, 3, 10, 40, 63):
        corr = np.sum(X[np.mod(r + d, n)] * tau)
        bf = np.sum(x * np.exp(-2j * np.pi * ((r - z / 2) * t / n + z * t * t / (2.0 * n * n))))
        assert abs(corr - bf) <= 1e-12 * abs(bf) + 1e-12


@pytest.mark.parametrize("z", [-40.0, -2.0, 2.0, 30.0])
def test_template_parseval_and_symmetry(z):
    """sum over all d of |tau_z(d)|^2 = int_0^1 |f|^2 = 1 (Parseval for the
    Fourier coefficients of a unit-modulus function); the tail beyond |d| = M
    decays like 1/(pi d)^2. And tau_{-z}(d) = conj(tau_z(-d))."""
    m = 1 << 14
    t = O.template_fresnel(z, m)
    s = np.sum(np.abs(t) ** 2)
    assert abs(s - 1.0) < 4.0 / (math.pi ** 2 * (m / 2 - abs(z)))
    tn = O.template_fresnel(-z, 512)
    tp = O.template_fresnel(z, 512)
    # index i <-> d = i - 256; -d <-> 512 - i (valid for i >= 1)
    assert np.max(np.abs(tn[1:] - np.conj(tp[1:][::-1]))) < 1e-14


def test_template_discrete_parseval_exact():
    n = 256
    t = O.template_discrete(14.0, n, n)
    assert abs(np.sum(np.abs(t) ** 2) - 1.0) < 1e-12


def test_z0_template_is_fourier_interpolation():
    """z = 0: integer offset gives tau = delta (plane row = |Xw|^2); a
    half-bin offset recovers the power of a tone lying halfway between bins
    (standard Fourier interpolation), which the bare bin underestimates by
    the scalloping factor 4/pi^2."""
    n = 4096
    f = 700.5
    t = np.arange(n)
    x = np.cos(2 * np.pi * f * t / n)
    X = O.spectrum(x)
    tau_half = O.template_fresnel(0.0, 256, offset=0.5)
    d = np.arange(-128, 128)
    r = 700
    a = np.sum(X[r + d] * tau_half)
    p_interp = abs(a) ** 2 / (n / 2) ** 2
    p_bin = abs(X[r]) ** 2 / (n / 2) ** 2
    assert abs(p_interp - 1.0) < 0.01
    assert abs(p_bin - 4 / math.pi ** 2) < 0.01
    assert np.array_equal(O.template_fresnel(0.0, 16), (np.arange(-8, 8) == 0).astype(complex))


# ----------------------------------------------------------------- plane --
def test_correlate_row_matches_direct_loop():
    """Steps 3-7 as a definition: the FFT correlation against plain loops,
    including both edges (zero outside [0, nb))."""
    rng = np.random.default_rng(5)
    nb, m = 40, 8
    Xw = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    tau = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    A = O.correlate_row(Xw, tau)
    for r in range(nb):
        acc = 0j
        for i in range(m):
            dd = i - m // 2
            if 0 <= r + dd < nb:
                acc += Xw[r + dd] * tau[i]
        assert abs(A[r] - acc) < 1e-12


def test_z0_row_of_plane_is_bin_power():
    rng = np.random.default_rng(6)
    Xw = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    taus = O.template_bank(10, 2, 32)
    P = O.power_plane(Xw, taus)
    zc = 5
    assert np.max(np.abs(P[zc] - np.abs(Xw) ** 2)) < 1e-12
    cells = O.plane_cells(Xw, taus, [0, 3, 10, 7], [0, 150, 299, 17])
    assert np.allclose(cells, P[[0, 3, 10, 7], [0, 150, 299, 17]], rtol=1e-12, atol=1e-12)


def test_noiseless_chirp_peaks_at_injected_cell():
    """An injected accelerated sinusoid (no noise, unit-noise normalisation)
    peaks on the grid next to (r0, z0); the true cell's brute-force chirped
    DFT power is s^2 (amplitude A = 2 s / sqrt(N))."""
    n = 1 << 17
    x = make_series(n, 1, [Chirp(10000.3, 35.0, 8.0, 0.3, 1)], noise=False,
                    dtype=np.float64)
    t = np.arange(n)
    bf = abs(np.sum(x * np.exp(-2j * np.pi * ((10000.3 - 17.5) * t / n
                                              + 35.0 * t * t / (2.0 * n * n))))) ** 2 / n
    assert abs(bf - 64.0) < 0.01
    X = O.spectrum(x) / math.sqrt(n)
    taus = O.template_bank(50, 2, 128)
    P = O.power_plane(X, taus)
    j, r = np.unravel_index(np.argmax(P), P.shape)
    assert r == 10000 and O.z_values(50, 2)[j] == 34.0
    # scalloping (0.3 bin) and a 1-unit z offset lose part of the power
    assert 40.0 < P[j, r] < 64.0
    # at an exactly on-grid signal the plane returns s^2 up to template truncation
    x2 = make_series(n, 1, [Chirp(10000.0, 34.0, 8.0, 0.3, 1)], noise=False,
                     dtype=np.float64)
    P2 = O.plane_cells(O.spectrum(x2) / math.sqrt(n), taus, [42], [10000])
    assert abs(P2[0] - 64.0) / 64.0 < 0.01


def test_cfg1_candidates_contain_injected_signal():
    x, p = workload("cfg1_n2e17_z50")
    Xw, taus, P, cands, _ = O.search(x, p["zmax"], p["dz"], p["m"], p["nharm"], p["sigma"])
    zs = O.z_values(p["zmax"], p["dz"])
    hits = [c for c in cands if c[2] == 1 and abs(c[0] - 10000) <= 1 and zs[c[1]] in (34.0, 36.0)]
    assert hits
    j, r = np.unravel_index(np.argmax(P), P.shape)
    assert abs(r - 10000) <= 1 and abs(zs[j] - 35.0) <= 2.0
    # whitened noise has unit mean power (median = ln 2 x mean for an exponential)
    assert 0.97 < np.mean(np.abs(Xw[1:]) ** 2) < 1.06


# ------------------------------------------------------------- whitening --
def test_whitening_brute_force_small():
    rng = np.random.default_rng(11)
    nb = 150
    X = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    Xw = O.whiten(X)
    p = [abs(v) ** 2 for v in X]
    assert Xw[0] == 0
    for k in range(1, nb):
        lo = k - 32
        if lo < 1:
            lo = 1
        if lo + 64 > nb:
            lo = nb - 64
        win = sorted(p[lo:lo + 64])
        mu = 0.5 * (win[31] + win[32])
        assert abs(Xw[k] - X[k] * math.sqrt(math.log(2) / mu)) < 1e-12


def test_whitening_constant_power_and_scale_invariance():
    nb = 500
    ph = np.exp(1j * np.linspace(0, 40, nb))
    Xw = O.whiten(3.0 * ph)
    assert np.allclose(np.abs(Xw[1:]) ** 2, math.log(2), rtol=1e-13)
    rng = np.random.default_rng(2)
    X = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    assert np.allclose(O.whiten(7.5 * X), O.whiten(X), rtol=1e-12, atol=1e-14)


# ------------------------------------------------------- half-bin planes --
@pytest.mark.parametrize("z", [0.0, 2.0, -2.0, 36.0, -50.0, 200.0])
def test_half_bin_template_matches_the_defining_integral(z):
    """tau_z(d) at offset 1/2 against adaptive quadrature of
    int_0^1 exp(2 pi i [(d - 1/2 + z/2) u - z u^2/2]) du."""
    from scipy import integrate
    m = 64 if abs(z) < 100 else 512
    tau = O.template_fresnel(z, m, offset=0.5)
    for d in (-m // 2, -7, -1, 0, 1, 5, m // 2 - 1):
        ph = lambda u: 2 * np.pi * ((d - 0.5 + z / 2) * u - z * u * u / 2)
        lim = 400 if abs(z) < 100 else 4000
        re = integrate.quad(lambda u: math.cos(ph(u)), 0, 1, limit=lim, epsabs=1e-13)[0]
        im = integrate.quad(lambda u: math.sin(ph(u)), 0, 1, limit=lim, epsabs=1e-13)[0]
        assert abs(tau[d + m // 2] - (re + 1j * im)) < 1e-10, (z, d)
    if z == 0.0:   # the Fourier interpolation kernel i / (pi (d - 1/2))
        d = np.arange(-m // 2, m // 2)
        assert np.allclose(tau, 1j / (np.pi * (d - 0.5)), atol=1e-15)


def test_half_bin_plane_recovers_a_half_bin_chirp():
    """A noiseless chirp midway between bins: the half-bin plane column
    2 r0 holds its full power s^2 (up to the m-tap truncation) at the true z,
    while the integer columns lose about 60% to scalloping."""
    n, s, r0, z0 = 1 << 14, 6.0, 2000.5, 20.0
    x = make_series(n, 0, [Chirp(r0, z0, s, 0.4, 1)], noise=False)
    Xw = O.spectrum(x) / math.sqrt(n)   # noiseless: unit-noise scaling, no whitening
    P2 = O.power_plane_interbin(Xw, 30, 2, 128)
    j0 = int((z0 + 30) // 2)
    assert abs(P2[j0, 2 * 2000 + 1] / s**2 - 1.0) < 0.03
    assert P2[j0, 4000] / s**2 < 0.5 and P2[j0, 4002] / s**2 < 0.5
    assert np.unravel_index(np.argmax(P2), P2.shape) == (j0, 4001)
    # the even columns are the integer plane
    P = O.power_plane(Xw, O.template_bank(30, 2, 128))
    assert np.array_equal(P2[:, 0::2], P)


# ------------------------------------------------------------ distillation --
@pytest.mark.parametrize("h", [1, 2, 4, 8, 16])
def test_log_gamma_tail_matches_library(h):
    from scipy import special
    for x in (0.5, 3.0, 17.0, 60.0, 200.0, 600.0):
        want = math.log(special.gammaincc(h, x))
        assert abs(O.log_gamma_tail(h, x) - want) <= 1e-11 * max(1.0, abs(want)), (h, x)


def test_sigma_of_the_thresholds_is_six():
    """T_h solves Q(h, T_h) = Phi_bar(6) (scipy's gammainccinv), so the
    significance of a sum exactly at T_h is 6 at every level."""
    T = O.thresholds(16, 6.0)
    for h, t in T.items():
        assert abs(O.gaussian_sigma(O.log_gamma_tail(h, t)) - 6.0) < 1e-8, h
    assert abs(O.gaussian_sigma(math.log(O.gaussian_tail(3.25))) - 3.25) < 1e-10


def test_sigma_far_tail_follows_the_asymptotic_series():
    """For h = 1, ln p = -x; at large x the Gaussian tail obeys
    ln Phi_bar(s) = -s^2/2 - ln(s sqrt(2 pi)) + ln(1 - 1/s^2 + 3/s^4 - 15/s^6 ...)."""
    for x in (2.0e3, 5.0e4, 1.0e6):
        s = O.gaussian_sigma(-x)
        series = -s * s / 2 - math.log(s * math.sqrt(2 * math.pi)) + \
            math.log(1 - 1 / s**2 + 3 / s**4 - 15 / s**6)
        assert abs(series + x) < 1e-6 * x, x
        assert s > math.sqrt(2 * x) * 0.95


def test_distill_brute_force_cases():
    Z = 21   # zc = 10
    # a 3x3 blob at level 1: only its maximum survives; a cell two bins away too
    blob = [(100 + dr, 10 + dj, 1, 25.0 + dr + 0.1 * dj) for dr in (-1, 0, 1) for dj in (-1, 0, 1)]
    far = [(103, 10, 1, 22.0)]
    out = O.distill(blob + far, Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(101, 11, 1), (103, 10, 1)]
    # a plateau: equal H, the smaller (j, r) wins
    out = O.distill([(50, 12, 2, 30.0), (51, 12, 2, 30.0), (50, 13, 2, 30.0)], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(50, 12, 2)]
    # across levels: the same signal at h = 1 (r, jc = 3) and h = 2 (2r + 1, 2 jc)
    lo = (200, 13, 1, 40.0)          # sigma ~ 8.5
    hi = (401, 16, 2, 60.0)
    out = O.distill([lo, hi], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(401, 16, 2)]
    hi_weak = (400, 16, 2, 30.0)
    out = O.distill([lo, hi_weak], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(200, 13, 1)]
    # the cross-level window is +-2 at the higher level, in the centred z
    # index: jc' = -3 and jc = -2 (|-3 + 4| = 1) match, jc = -3 (distance 3)
    # does not, nor does r' = 2r + 3
    out = O.distill([(300, 7, 2, 80.0), (150, 8, 1, 30.0)], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(300, 7, 2)]
    out = O.distill([(300, 7, 2, 80.0), (150, 7, 1, 30.0)], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(150, 7, 1), (300, 7, 2)]
    out = O.distill([(303, 10, 2, 80.0), (150, 10, 1, 30.0)], Z)
    assert len(out) == 2
    out = O.distill([(302, 12, 2, 80.0), (151, 10, 1, 30.0), (150, 11, 1, 29.0)], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(302, 12, 2)]
    # the window is 8-connected: a diagonal neighbour alone suppresses
    out = O.distill([(100, 10, 1, 25.0), (101, 11, 1, 30.0)], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(101, 11, 1)]
    # across levels sigma decides, not H: H = 26 at h = 2 is less
    # significant than H = 25 at h = 1
    assert O.gaussian_sigma(O.log_gamma_tail(2, 26.0)) < O.gaussian_sigma(-25.0)
    out = O.distill([(200, 13, 1, 25.0), (400, 16, 2, 26.0)], Z)
    assert [(r, j, h) for (r, j, h, *_) in out] == [(200, 13, 1)]
    # sigma and log10 p of a survivor
    (r, j, h, H, sig, l10) = O.distill([(10, 10, 4, 40.0)], Z)[0]
    from scipy import special, stats
    assert abs(l10 - math.log10(special.gammaincc(4, 40.0))) < 1e-10
    assert abs(sig - stats.norm.isf(special.gammaincc(4, 40.0))) < 1e-8


# ------------------------------------------------- block-median whitening --
def test_block_median_brute_force_small():
    """Sorted-list medians of each block and the two-point interpolation
    formula, written out with loops, on a spectrum whose last block is short."""
    rng = np.random.default_rng(31)
    nb = 64 * 5 + 18
    X = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    p = [abs(v) ** 2 for v in X]
    meds, cens = [], []
    a = 1
    while a < nb:
        b = min(a + 64, nb)
        vals = sorted(p[a:b])
        c = len(vals)
        meds.append(vals[c // 2] if c % 2 else 0.5 * (vals[c // 2 - 1] + vals[c // 2]))
        cens.append((a + b - 1) / 2.0)
        a = b
    assert len(meds) == 6 and cens[-1] == (321 + 337) / 2.0
    mu = O.block_median_power(X)
    for k in range(1, nb):
        if k <= cens[0]:
            want = meds[0]
        elif k >= cens[-1]:
            want = meds[-1]
        else:
            i = max(i for i in range(len(cens)) if cens[i] <= k)
            t = (k - cens[i]) / (cens[i + 1] - cens[i])
            want = (1 - t) * meds[i] + t * meds[i + 1]
        assert abs(mu[k] - want) <= 1e-12 * want, k
    Xw = O.whiten_block(X)
    assert Xw[0] == 0
    assert np.allclose(np.abs(Xw[1:]) ** 2, np.array(p[1:]) * math.log(2) / mu[1:], rtol=1e-12)


def test_block_median_linear_ramp_is_exact():
    """A power ramp a + b k has each block median at its centre, so the
    interpolation reproduces it exactly between the first and last centre and
    the whitened power there is ln 2 (any plausible slip in the centres or the
    interpolation breaks this)."""
    nb = 64 * 9 + 40
    k = np.arange(nb)
    pw = 3.0 + 0.25 * k
    X = np.sqrt(pw) * np.exp(1j * 0.37 * k)
    mu = O.block_median_power(X)
    inner = (k >= 32.5) & (k <= (1 + 64 * 9 + nb - 1) / 2.0)
    assert np.allclose(mu[inner], pw[inner], rtol=1e-13)
    assert np.allclose(mu[1:33], pw[32] + 0.125, rtol=1e-13)   # first centre 32.5
    Xw = O.whiten_block(X)
    assert np.allclose(np.abs(Xw[inner]) ** 2, math.log(2), rtol=1e-12)


def test_block_median_constant_power_and_scale_invariance():
    rng = np.random.default_rng(8)
    nb = 4096 + 7
    ph = np.exp(2j * np.pi * rng.random(nb))
    Xw = O.whiten_block(2.5 * ph)
    assert np.allclose(np.abs(Xw[1:]) ** 2, math.log(2), rtol=1e-12)
    X = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    assert np.allclose(O.whiten_block(4.0 * X), O.whiten_block(X), rtol=1e-12, atol=1e-14)
    # whitened noise has unit mean power
    X = rng.standard_normal(1 << 18) + 1j * rng.standard_normal(1 << 18)
    assert abs(np.mean(np.abs(O.whiten_block(X)[1:]) ** 2) - 1.0) < 0.02


def test_whitening_rejects_short_spectrum():
    with pytest.raises(ValueError):
        O.whiten(np.ones(64, dtype=complex))


# ------------------------------------------------------- harmonic sums --
def test_subharmonic_rounding_rules():
    # round half up in r
    assert list(O.subharmonic_r([0, 1, 2, 3, 5, 7], 1, 2)) == [0, 1, 1, 2, 3, 4]
    assert list(O.subharmonic_r([8, 9, 10], 3, 4)) == [6, 7, 8]
    # ties away from zero in the centred z index, symmetric about zc
    zc = 10
    assert list(O.subharmonic_j([9, 11, 7, 13], 1, 2, zc)) == [9, 11, 8, 12]
    assert list(O.subharmonic_j([10], 5, 16, zc)) == [10]


def test_harmonic_sum_invariants():
    Z, nb = 21, 200
    zc = 10
    # constant plane: H_h = h c
    H = O.harmonic_sums(np.full((Z, nb), 2.5), 16)
    for h, v in H.items():
        assert np.allclose(v, 2.5 * h)
    # plane = column index: at r = h t, H_h = sum_k k t = t h (h+1) / 2
    P = np.tile(np.arange(nb, dtype=float), (Z, 1))
    H = O.harmonic_sums(P, 16)
    for h in (1, 2, 4, 8, 16):
        for t in (1, 3, 12):
            r = h * t
            if r < nb:
                assert H[h][4, r] == t * h * (h + 1) / 2
    # plane = centred row index: at jc = h t, H_h = sum_k k t
    P = np.tile((np.arange(Z) - zc)[:, None].astype(float), (1, nb))
    H = O.harmonic_sums(P, 8)
    for h in (1, 2, 4, 8):
        for t in (-1, 1):
            j = zc + h * t
            if 0 <= j < Z:
                assert H[h][j, 50] == t * h * (h + 1) / 2
    # z-mirror symmetry of the plane carries over to the sums
    rng = np.random.default_rng(0)
    half = rng.random((zc + 1, nb))
    P = np.vstack([half[:0:-1], half])
    H = O.harmonic_sums(P, 16)
    for v in H.values():
        assert np.allclose(v, v[::-1])


def test_harmonic_sum_brute_force_hot_cell():
    """A single unit cell at (j0, r0) appears in H_h exactly at the top cells
    whose k-th sub-harmonic lands on it; counted here by brute force."""
    Z, nb = 17, 120
    zc = 8
    j0, r0 = 9, 7
    P = np.zeros((Z, nb))
    P[j0, r0] = 1.0
    H = O.harmonic_sums(P, 16)
    for h in (1, 2, 4, 8, 16):
        for j in range(Z):
            for r in range(nb):
                cnt = 0
                for k in range(1, h + 1):
                    rr = math.floor(k * r / h + 0.5)
                    jc = j - zc
                    x = k * jc / h
                    jj = zc + int(math.copysign(math.floor(abs(x) + 0.5), x))
                    cnt += (rr == r0 and jj == j0)
                assert H[h][j, r] == cnt
    assert H[2][zc + 2 * (j0 - zc), 2 * r0] >= 1


# ------------------------------------------------------------- thresholds --
def test_thresholds_closed_forms():
    p = O.gaussian_tail(6.0)
    assert abs(p - 9.865876450377e-10) < 1e-20
    T = O.thresholds(16, 6.0)
    assert abs(T[1] + math.log(p)) < 1e-10           # Gamma(1) is exponential
    for h, t in T.items():
        # Poisson form of the upper tail of Gamma(h, 1) for integer h
        q = math.exp(-t) * sum(t ** i / math.factorial(i) for i in range(h))
        assert abs(q / p - 1.0) < 1e-9


def test_threshold_false_alarm_rate_monte_carlo():
    """At 2 sigma the false-alarm rate of sums of h unit exponentials at T_h
    matches the Gaussian tail (so the thresholds have the right meaning)."""
    rng = np.random.default_rng(7)
    T = O.thresholds(16, 2.0)
    p = O.gaussian_tail(2.0)
    for h, t in T.items():
        s = rng.exponential(size=(400000, h)).sum(axis=1)
        rate = np.mean(s >= t)
        assert abs(rate - p) < 5 * math.sqrt(p / 400000)


def test_thresholds_golden_table():
    with open(os.path.join(GOLDEN, "thresholds_sigma6.json")) as f:
        g = json.load(f)
    T = O.thresholds(16, 6.0)
    for h, v in g["T"].items():
        assert abs(T[int(h)] - v) < 1e-9


# ------------------------------------------- windowed sums, cells, candidates --
def _brute_H(P, h, j, r):
    """H_h(r, j) by explicit loops over k with the rounding rules spelled out
    in real arithmetic (round half up in r, half away from zero in jc)."""
    Z = P.shape[0]
    zc = (Z - 1) // 2
    s = 0.0
    for k in range(1, h + 1):
        rr = math.floor(k * r / h + 0.5)
        x = k * (j - zc) / h
        jj = zc + int(math.copysign(math.floor(abs(x) + 0.5), x))
        s += P[jj, rr]
    return s


def _small_whitened(nb, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) / math.sqrt(2.0)


def test_correlate_band_equals_direct_sums_at_both_edges():
    """A column range of Eq. 1 through a sub-band FFT equals the direct sums
    sum_d Xw[r+d] tau(d), including ranges that reach past either end of the
    spectrum (where Xw is zero)."""
    nb, m = 300, 16
    Xw = _small_whitened(nb, 11)
    taus = O.template_bank(6, 2, m)
    for c0, c1 in ((0, 40), (5, 6), (130, 171), (270, 300), (0, 300)):
        for j in (0, 3, 6):
            got = np.abs(O.correlate_band(Xw, taus[j], c0, c1)) ** 2
            ref = O.plane_cells(Xw, taus, np.full(c1 - c0, j), np.arange(c0, c1))
            assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, ref.max())


def test_harmonic_sums_window_equals_whole_plane_sums():
    """Windowed sums (the plane formed only at the columns each ratio k/h
    reads) equal the whole-plane sums restricted to the window, at the start,
    in the middle and at the end of the spectrum, for every level."""
    nb, m, zmax = 700, 16, 8
    Xw = _small_whitened(nb, 12)
    taus = O.template_bank(zmax, 2, m)
    H = O.harmonic_sums(O.power_plane(Xw, taus), 16)
    for r_a, r_b in ((0, 37), (301, 420), (650, 700)):
        Hw = O.harmonic_sums_window(Xw, taus, 16, r_a, r_b)
        assert sorted(Hw) == [1, 2, 4, 8, 16]
        for h in Hw:
            assert np.max(np.abs(Hw[h] - H[h][:, r_a:r_b])) <= 1e-10 * H[h].max()


def test_harmonic_sum_cells_equals_brute_force():
    """harmonic_sum_cells (direct Eq. 1 cell sums) against the loop-defined
    H_h on the whole oracle plane, at random cells including both z edges
    and the lowest bins; (j, r) swapped anywhere would fail it."""
    nb, m, zmax = 400, 16, 10
    Xw = _small_whitened(nb, 13)
    taus = O.template_bank(zmax, 2, m)
    P = O.power_plane(Xw, taus)
    Z = taus.shape[0]
    rng = np.random.default_rng(5)
    js = np.concatenate([[0, Z - 1, 2, Z - 3], rng.integers(0, Z, 40)])
    rs = np.concatenate([[1, 399, 3, 17], rng.integers(1, nb, 40)])
    got = O.harmonic_sum_cells(Xw, taus, 16, js, rs)
    for h in (1, 2, 4, 8, 16):
        ref = np.array([_brute_H(P, h, j, r) for j, r in zip(js, rs)])
        assert np.max(np.abs(got[h] - ref)) <= 1e-10 * max(1.0, ref.max()), h


def test_candidates_equal_brute_force_list():
    """candidates() against an explicit loop over h, then r >= 1, then j,
    that keeps (r, j, h, H) with H >= T_h: the same rows in the same order.
    At sigma = 1 the thresholds are low enough for many rows at every level;
    planted cells put H exactly on T_1 (kept) and one float below (dropped),
    and a large bin-0 column checks that r = 0 is never a candidate."""
    rng = np.random.default_rng(9)
    Z, nb = 9, 160
    P = rng.exponential(size=(Z, nb))
    T = O.thresholds(16, 1.0)
    P[:, 0] = 50.0
    P[2, 40] = T[1]
    P[3, 41] = np.nextafter(T[1], 0.0)
    rows, H = O.candidates(P, 16, 1.0)
    want = []
    for h in (1, 2, 4, 8, 16):
        for r in range(1, nb):
            for j in range(Z):
                v = _brute_H(P, h, j, r)
                if v >= T[h]:
                    want.append((r, j, h, v))
    assert [(a, b, c) for a, b, c, _ in rows] == [(a, b, c) for a, b, c, _ in want]
    assert np.allclose([v for *_, v in rows], [v for *_, v in want], rtol=1e-12, atol=0)
    keys = {(a, b, c) for a, b, c, _ in rows}
    assert (40, 2, 1) in keys and (41, 3, 1) not in keys
    assert all(r >= 1 for r, *_ in rows)
    assert {c for _, _, c, _ in rows} == {1, 2, 4, 8, 16}
