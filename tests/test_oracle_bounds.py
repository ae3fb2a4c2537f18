"""Pins of oracle/bounds.py (Section 3, Theorems 2 and 4; Appendix B, Lemmas
dbound and qbound; Theorem 1's rank rule) against values worked out by hand.

The case: two points whose kernel value is a = 1/4, so K = [[1, a], [a, 1]],
and the Nystrom approximation from the first column (Section 1.2),
K~ = K(:,0) K(0,0)^-1 K(0,:) = [[1, a], [a, a^2]].  K - K~ = diag(0, 1 - a^2)
is positive semidefinite.  Every quantity the bounds use is a small rational
(or one square root), derived by hand:

  d = K 1 = (5/4, 5/4)            d~ = K~ 1 = (5/4, 5/16)
  q = K D^-1 1 = (1, 1)           q~ = K~ D~^-1 1 = (8/5, 2/5)
  tr K = 2, tr(K - K~) = 15/16, |K| = 5/4 (eigenvalues 1 +- a)
  d_min = 5/4, delta = delta_d = 5/16, q_min = 1, delta_q = 2/5
  G~ = Q~^-1/2 K~ D~^-1 has equal columns (alpha, beta), alpha^2 = 2/5,
       beta^2 = 1/10, so |G~| = sqrt(2 (alpha^2 + beta^2)) = 1
  L - L~ = [[0, a - sqrt a], [a - sqrt a, 1 - a]] / (1 + a): trace norm
       sqrt((1 - a)^2 + 4 (a - sqrt a)^2) / (1 + a) = sqrt(13) / 5
  P = D^-1 K Q^-1 K D^-1 = [[17, 8], [8, 17]] / 25, P~ = G~^T G~ = [[1, 1], [1, 1]] / 2,
       P - P~ = (9/50) [[1, -1], [-1, 1]]: trace norm 9/25

The bound values are the paper's expressions evaluated at these hand-derived
ingredients; a dropped sqrt(N), a d_min where delta_d belongs, a q_min where
delta_q belongs, or (1 + |G~|) squared each moves them.
"""
import math

import numpy as np

from oracle import bounds

A = 0.25
K = np.array([[1.0, A], [A, 1.0]])
KT = np.array([[1.0, A], [A, A * A]])
TR = 15.0 / 16.0          # tr(K - K~)
SQN = math.sqrt(2.0)      # sqrt(N)


def test_trace_norm_closed_form():
    assert abs(bounds.trace_norm(np.diag([3.0, -2.0, 0.5])) - 5.5) < 1e-15


def test_lemma_dbound_hand_values():
    mx, bmx, ss, bss = bounds.lemma_dbound(K, KT)
    assert abs(mx - 15.0 / 16.0) < 1e-15                 # |5/4 - 5/16|
    assert abs(bmx - SQN * TR) < 1e-15
    assert abs(ss - 225.0 / 256.0) < 1e-15
    assert abs(bss - 2.0 * TR * TR) < 1e-15


def test_lemma_qbound_hand_values():
    mx, b = bounds.lemma_qbound(K, KT)
    assert abs(mx - 3.0 / 5.0) < 1e-15                   # q - q~ = (-3/5, 3/5)
    # sqrt(N) / delta_d (1 + |K| / delta_d) tr(K - K~) = sqrt2 * 16/5 * 5 * 15/16 = 15 sqrt2
    assert abs(b - 15.0 * SQN) < 1e-12


def test_theorem2_hand_values():
    err, b = bounds.theorem2_bound(K, KT)
    assert abs(err - math.sqrt(13.0) / 5.0) < 1e-14
    d_min, delta, trk = 5.0 / 4.0, 5.0 / 16.0, 2.0
    want = (1.0 / d_min + SQN / delta ** 2 * trk + 2.0 / (4.0 * delta ** 3) * trk * TR) * TR
    assert abs(want - 56.7029003976) < 1e-9               # the same number written out
    assert abs(b - want) < 1e-10 * want


def test_theorem4_hand_values():
    err, b = bounds.theorem4_bound(K, KT)
    assert abs(err - 9.0 / 25.0) < 1e-14
    d_min, q_min, dd, dq, trk, normk, normg = 5.0 / 4.0, 1.0, 5.0 / 16.0, 2.0 / 5.0, 2.0, 5.0 / 4.0, 1.0
    br = (1.0 / (math.sqrt(q_min) * d_min) + SQN * trk / (math.sqrt(dq) * dd ** 2)
          + SQN * trk / (2.0 * dq ** 1.5 * dd ** 2) * (1.0 + normk / dd))
    want = (1.0 + normg) * br * TR
    assert abs(want - 624.0213249359) < 1e-8
    assert abs(b - want) < 1e-10 * want


def test_bounds_hold_on_hand_case():
    for f in (bounds.theorem2_bound, bounds.theorem4_bound, bounds.lemma_qbound):
        err, b = f(K, KT)
        assert err <= b


def test_theorem1_rank_and_best_rank_error():
    # r'/eps + r' log(1/(eps eta)) at r' = 10, eps = 1/2, eta = 1/10: 20 + 10 log 20
    assert abs(bounds.theorem1_rank(10, 0.5, 0.1) - (20.0 + 10.0 * math.log(20.0))) < 1e-12
    Q = np.linalg.qr(np.random.Generator(np.random.PCG64(4)).standard_normal((4, 4)))[0]
    Kd = (Q * np.array([3.0, 2.0, 1.0, 0.5])) @ Q.T
    assert abs(bounds.best_rank_error(Kd, 1) - 3.5) < 1e-12
    assert abs(bounds.best_rank_error(Kd, 3) - 0.5) < 1e-12
