"""The transit kernel's rearrangements of the geometry, written out in FP64
and checked against the oracle's plain definitions (Sec. 6.1, the transit
recipe; hydrostatic radii with g ~ r^-2 anchored at P_ref):

* altitudes instead of radii: r = 1 / (1/R_p + C phi) becomes
  z = r - R_p = -C phi R_p^2 / (1 + C phi R_p), without the cancellation of
  r - R_p;
* chords from altitude differences: ds_ik = 2 (sqrt A - sqrt B) with
  A = r_k^2 - b^2 = (z_k - z_b)(2 R_p + z_k + z_b) and B likewise for
  r_{k+1}, computed as 2 (A - B) / (sqrt A + sqrt B) with
  A - B = (z_k - z_{k+1})(2 R_p + z_k + z_{k+1});
* the trapezoid in impact parameter regrouped per ray:
  sum_i (f_i r_i + f_{i+1} r_{i+1}) (r_i - r_{i+1}) / 2
    = sum_{i>=1} f_i r_i (z_{i-1} - z_{i+1}) / 2  (z_L := z_{L-1}),
  ray 0 grazing the top level with tau = 0;
* 1 - e^-tau by its six-term series below tau = 1/8 (truncation below
  tau^6 / 7! = 7.6e-10 relative).
Each is an identity (or a negligible truncation), so the restated depth
agrees with the oracle's to rounding."""
import numpy as np

from oracle import transmission as Tr
from oracle.constants import K_BOLTZ, AMU, BAR

G = 2182.73


def _one_minus_exp(tau):
    s = 1.0 - tau / 6.0
    s = 1.0 - tau * 0.2 * s
    s = 1.0 - tau * 0.25 * s
    s = 1.0 - tau / 3.0 * s
    s = 1.0 - tau * 0.5 * s
    series = tau * s
    return np.where(tau < 0.125, series, -np.expm1(-tau))


def test_one_minus_exp_series():
    tau = np.geomspace(1e-12, 0.125, 2000)
    assert np.max(np.abs(_one_minus_exp(tau) / -np.expm1(-tau) - 1)) < 1e-9


def test_restated_transit_depth_equals_the_oracle():
    rng = np.random.default_rng(5)
    for L, mu in ((40, 2.3), (150, 2.3), (97, 2.6)):
        p = np.logspace(-8, 2, L)
        T = rng.uniform(700.0, 2300.0, L)
        rp, rs = 1.21 * 7.1492e9, 0.9 * 6.957e10
        r_ref = Tr.radii(p, T, rp, 0.1, G, mu)
        # altitudes from the same hydrostatic integral, phi relative to P_ref
        cphi = 1.0 / r_ref - 1.0 / rp                      # = C phi
        z = -cphi * rp * rp / (1.0 + cphi * rp)
        assert np.max(np.abs((rp + z) / r_ref - 1)) < 1e-14
        rho = p * BAR * mu * AMU / (K_BOLTZ * T)
        chi = 10 ** rng.uniform(-6, 2, (L, 5))
        alpha = chi * rho[:, None]
        abar = 0.5 * (alpha[:-1] + alpha[1:])
        integ = np.zeros(5)
        for i in range(1, L):
            zb = z[i]
            k = np.arange(i)
            A = (z[k] - zb) * (2 * rp + z[k] + zb)
            B = np.where(k + 1 < i, (z[k + 1] - zb) * (2 * rp + z[k + 1] + zb), 0.0)
            AmB = (z[k] - z[k + 1]) * (2 * rp + z[k] + z[k + 1])
            ds = 2.0 * AmB / (np.sqrt(A) + np.sqrt(np.maximum(B, 0.0)))
            tau = ds @ abar[:i]
            wgt = 0.5 * (z[i - 1] - (z[i + 1] if i + 1 < L else z[i]))
            integ += _one_minus_exp(tau) * (rp + zb) * wgt
        got = ((rp + z[-1]) / rs) ** 2 + 2.0 * integ / rs ** 2
        ref = Tr.transit_depth(chi, p, T, r_ref, rs, mu)
        assert np.max(np.abs(got / ref - 1)) < 1e-11, (L, np.max(np.abs(got / ref - 1)))
