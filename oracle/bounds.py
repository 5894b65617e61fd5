"""Bias bounds for reduced-precision Metropolis-Hastings (Sec. 3 and App. C), in FP64.

* TV distance (Eq. tv): ||pi - pi~||_TV = 1/2 sum_x |pi(x) - pi~(x)|.
* Perturbed target (Eq. pi tilde def): pi~ = pi exp(delta) / Z.
* Observable bias (Eq. bias_gaussian): |E_pi~ f - E_pi f| <= 2 A ||pi - pi~||_TV for |f| <= A.
* Gaussian delta with std sigma: KL = sigma^2 / 2 and, by Pinsker, TV <= sigma / 2 (Eq. tv_gaussian).
* Acceptance error (Step 3 of the proof of Theorem 2):
  |min{1, s e^eps} - min{1, s}| <= 1 - exp(-|eps|).
* Theorem 2: ||pi'(P~ - P)||_TV <= 1 - E_{x ~ pi', y ~ q}[exp(-|eps(x, y)|)].
* Theorem 1: ||pi~ - pi||_TV <= ||pi~(P~ - P)||_TV / (1 - r).
* Theorem 3 (Eq. avg_bound), eps ~ N(mu, 2 sigma^2), local proposal:
  TV <= (1 - e^{sigma^2}/2 [e^{-mu} erfc(sigma - mu/(2 sigma)) + e^{mu} erfc(sigma + mu/(2 sigma))]) / (1 - r).
* mu = 0 form (Eq. tvmuzero): TV <= (1 - e^{sigma^2} erfc(sigma)) / (1 - r).
The text after Eq. tvmuzero says the mu = 0 bound scales as sigma^2; expanding it
gives 2 sigma / sqrt(pi) + O(sigma^2), so it is linear in sigma.  The formula is
implemented as printed and the bound reported is min(Pinsker, Theorem 3) at
r = 0, as in the paper's Fig. 1(b) and Fig. 3(b).
"""
import numpy as np
from scipy.special import erfc


def tv_distance(p, q):
    return 0.5 * np.abs(np.asarray(p) - np.asarray(q)).sum()


def perturbed_pi(pi, delta):
    w = np.asarray(pi) * np.exp(np.asarray(delta) - np.max(delta))
    return w / w.sum()


def pinsker_bound(sigma):
    return 0.5 * np.asarray(sigma, dtype=np.float64)


def kl_gaussian(sigma):
    return 0.5 * np.asarray(sigma, dtype=np.float64) ** 2


def delta_alpha(s, eps):
    s = np.asarray(s, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    return np.abs(np.minimum(1.0, s * np.exp(eps)) - np.minimum(1.0, s))


def delta_alpha_bound(eps):
    return 1.0 - np.exp(-np.abs(np.asarray(eps, dtype=np.float64)))


def thm2_bound(eps):
    """1 - mean(exp(-|eps|)) over proposals drawn as x ~ pi', y ~ q(.|x)."""
    return 1.0 - np.mean(np.exp(-np.abs(np.asarray(eps, dtype=np.float64))))


def thm1_rhs(pi_t, P_t, P, r):
    return tv_distance(0.0, pi_t @ (P_t - P)) / (1.0 - r)


def thm3_bound(mu, sigma, r=0.0):
    mu = float(mu)
    sigma = float(sigma)
    if sigma == 0.0:
        return (1.0 - np.exp(-abs(mu))) / (1.0 - r)
    bracket = (np.exp(-mu) * erfc(sigma - mu / (2.0 * sigma))
               + np.exp(mu) * erfc(sigma + mu / (2.0 * sigma)))
    return (1.0 - 0.5 * np.exp(sigma ** 2) * bracket) / (1.0 - r)


def thm3_mu0_bound(sigma, r=0.0):
    return (1.0 - np.exp(sigma ** 2) * erfc(sigma)) / (1.0 - r)


def reported_bound(mu, sigma_eps_std):
    """min(Pinsker, Theorem 3) at r = 0 from the measured increments eps ~ N(mu, 2 sigma^2):
    sigma = std(eps) / sqrt(2) is the std of delta."""
    sigma = float(sigma_eps_std) / np.sqrt(2.0)
    return min(float(pinsker_bound(sigma)), thm3_bound(mu, sigma))


UNIT_ROUNDOFF = {
    # App. A, Table tab:precision.  The table prints 4.88e-5 for f16; the f16 format
    # (10 explicit significand bits) has unit roundoff 2^-11 = 4.88e-4, which is used here.
    "bf16": 2.0 ** -8,
    "f16": 2.0 ** -11,
    "f32": 2.0 ** -24,
    "f64": 2.0 ** -53,
}
