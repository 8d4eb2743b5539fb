"""Pins for the theta control (Alg. 1's Theta_Estimation / OPT_Lower_Bound /
Set_Theta, defined by Tang, Shi & Xiao, SIGMOD 2015).  Each constant is checked
against the bound it is derived from, not against its own closed form."""
import math

import pytest

import oracle

CASES = [(4096, 10, 0.5, 1.0), (1 << 20, 50, 0.13, 1.0), (1 << 22, 100, 0.5, 1.0),
         (1000, 1, 0.3, 1.0), (65536, 200, 0.1, 2.0), (3, 2, 0.4, 1.0)]


@pytest.mark.parametrize("n,k,eps,ell", CASES)
def test_ln_binomial_exact(n, k, eps, ell):
    # ln C(n, k) against the exact big-integer binomial
    prm = oracle.theta_params(n, k, eps, ell)
    exact = math.log(math.comb(n, k))
    assert abs(prm["lnC"] - exact) <= 1e-12 * max(1.0, exact) * k


@pytest.mark.parametrize("n,k,eps,ell", CASES)
def test_ell_prime_splits_failure_probability(n, k, eps, ell):
    # ell' is chosen so that n^-ell' = n^-ell / 2^ell: the two phases each fail
    # with probability at most half the overall budget (for ell = 1)
    prm = oracle.theta_params(n, k, eps, ell)
    lhs = -prm["ell_p"] * math.log(n)
    rhs = -ell * math.log(n) - ell * math.log(2.0)
    assert abs(lhs - rhs) < 1e-9 * abs(rhs)


@pytest.mark.parametrize("n,k,eps,ell", CASES)
def test_lambda_star_balances_both_bounds(n, k, eps, ell):
    # Tang et al. Sec. 3: the optimal seed set is estimated within (1-eps1) when
    #   theta >= 2 n ln(1/delta1) / (OPT eps1^2),
    # and greedy is (1-1/e-eps)-approximate when
    #   theta >= (2-2/e) n ln(C(n,k)/delta2) / (OPT (eps - (1-1/e) eps1)^2),
    # with delta1 = delta2 = n^-ell' / 2.  lambda* is OPT times the common value
    # of both bounds at the eps1 that equalises them.
    prm = oracle.theta_params(n, k, eps, ell)
    lp = prm["ell_p"]
    ln_inv_delta = lp * math.log(n) + math.log(2.0)
    lnC = math.log(math.comb(n, k))
    g = 1.0 - 1.0 / math.e

    def b1(e1):
        return 2.0 * n * ln_inv_delta / e1 ** 2

    def b2(e1):
        return (2.0 - 2.0 / math.e) * n * (lnC + ln_inv_delta) / (eps - g * e1) ** 2

    # solve b1 = b2 for eps1 in (0, eps/g) by bisection
    lo, hi = 1e-12, eps / g * (1 - 1e-12)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if b1(mid) > b2(mid):
            lo = mid
        else:
            hi = mid
    e1 = 0.5 * (lo + hi)
    want = b1(e1)
    assert abs(prm["lambda_star"] - want) < 1e-9 * want
    # and no other eps1 gives a smaller requirement
    for t in (0.9, 0.99, 1.01, 1.1):
        assert max(b1(e1 * t), b2(e1 * t)) >= want * (1 - 1e-12)


@pytest.mark.parametrize("n,k,eps,ell", CASES)
def test_lambda_prime_solves_martingale_tail(n, k, eps, ell):
    # Tang et al. Sec. 4 (OPT lower bound): with theta_i = lambda'/x sets and
    # every seed set's coverage mean at most x/n, the martingale tail bound
    #   Pr[sum - theta p >= d theta p] <= exp(-d^2 theta p / (2 + 2d/3)),
    # at d = eps', p = x/n, must fall to n^-ell' / (C(n,k) log2 n).
    prm = oracle.theta_params(n, k, eps, ell)
    if n < 4:
        return
    ep = prm["eps_p"]
    assert abs(ep - math.sqrt(2.0) * eps) < 1e-15
    lnC = math.log(math.comb(n, k))
    target = -(prm["ell_p"] * math.log(n) + lnC + math.log(math.log2(n)))
    for i in range(1, 6):
        x = n / 2.0 ** i
        theta = prm["lambda_prime"] / x
        log_tail = -ep ** 2 * theta * (x / n) / (2.0 + 2.0 * ep / 3.0)
        assert abs(log_tail - target) < 1e-9 * abs(target)


def test_round_count():
    # loop bound i = 1 .. ceil(log2 n) - 1
    assert oracle.theta_params(4096, 10, 0.5, 1.0)["rounds"] == 11
    assert oracle.theta_params(4097, 10, 0.5, 1.0)["rounds"] == 12
    assert oracle.theta_params(2, 1, 0.5, 1.0)["rounds"] == 0


def test_ladder_first_round_values():
    # first-round theta = ceil(2 lambda' / n) for the three plain workloads
    # (2 lambda'/n = 786.5, 70612.4, 11667.2: each rounds up)
    for (n, k, eps, want) in [(4096, 10, 0.5, 787), (1 << 20, 50, 0.13, 70613),
                              (1 << 22, 100, 0.5, 11668)]:
        prm = oracle.theta_params(n, k, eps, 1.0)
        assert math.ceil(prm["lambda_prime"] / (n / 2.0)) == want
