"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in the CPU oracle's Lemma 3-6 code (a dropped
term, swapped operands, a transposed factor, a sign) through monkeypatch and
checks that at least one pin test then fails.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import lemmas as L
import test_oracle_pins as P

inv = np.linalg.inv


def m_combine_drop_C_eta(ai, aj):
    n = ai.A.shape[0]; I = np.eye(n)
    M1 = inv(I + ai.C @ aj.J); M2 = inv(I + aj.J @ ai.C)
    return L.FElem(aj.A @ M1 @ ai.A, aj.A @ M1 @ ai.b + aj.b,
                   aj.A @ M1 @ ai.C @ aj.A.T + aj.C,
                   ai.A.T @ M2 @ (aj.eta - aj.J @ ai.b) + ai.eta,
                   ai.A.T @ M2 @ aj.J @ ai.A + ai.J)


def m_combine_swapped_M(ai, aj):
    n = ai.A.shape[0]; I = np.eye(n)
    M1 = inv(I + aj.J @ ai.C); M2 = inv(I + ai.C @ aj.J)
    return L.FElem(aj.A @ M1 @ ai.A, aj.A @ M1 @ (ai.b + ai.C @ aj.eta) + aj.b,
                   aj.A @ M1 @ ai.C @ aj.A.T + aj.C,
                   ai.A.T @ M2 @ (aj.eta - aj.J @ ai.b) + ai.eta,
                   ai.A.T @ M2 @ aj.J @ ai.A + ai.J)


def m_combine_eta_sign(ai, aj):
    n = ai.A.shape[0]; I = np.eye(n)
    M1 = inv(I + ai.C @ aj.J); M2 = inv(I + aj.J @ ai.C)
    return L.FElem(aj.A @ M1 @ ai.A, aj.A @ M1 @ (ai.b + ai.C @ aj.eta) + aj.b,
                   aj.A @ M1 @ ai.C @ aj.A.T + aj.C,
                   ai.A.T @ M2 @ (aj.eta + aj.J @ ai.b) + ai.eta,
                   ai.A.T @ M2 @ aj.J @ ai.A + ai.J)


def m_combine_drop_Cj(ai, aj):
    n = ai.A.shape[0]; I = np.eye(n)
    M1 = inv(I + ai.C @ aj.J); M2 = inv(I + aj.J @ ai.C)
    return L.FElem(aj.A @ M1 @ ai.A, aj.A @ M1 @ (ai.b + ai.C @ aj.eta) + aj.b,
                   aj.A @ M1 @ ai.C @ aj.A.T,
                   ai.A.T @ M2 @ (aj.eta - aj.J @ ai.b) + ai.eta,
                   ai.A.T @ M2 @ aj.J @ ai.A + ai.J)


_orig_fe = L.filter_element


def m_element_drop_F(F, u, Q, H, d, R, y):
    e = _orig_fe(F, u, Q, H, d, R, y)
    n = F.shape[0]
    S = H @ Q @ H.T + R
    K = Q @ H.T @ inv(S)
    return e._replace(A=(np.eye(n) - K @ H))


_orig_se = L.smoother_element


def m_selem_drop_u(F, u, Q, xbar, P):
    return _orig_se(F, np.zeros_like(u), Q, xbar, P)


def m_selem_L_sign(F, u, Q, xbar, P):
    e = _orig_se(F, u, Q, xbar, P)
    return e._replace(L=P + e.E @ F @ P)


def m_scomb_transpose(ai, aj):
    return L.SElem(ai.E @ aj.E, ai.E @ aj.g + ai.g, ai.E.T @ aj.L @ ai.E + ai.L)


def m_scomb_swap(ai, aj):
    return L.SElem(aj.E @ ai.E, aj.E @ ai.g + aj.g, aj.E @ ai.L @ aj.E.T + aj.L)


def m_suffix_reversed_prefix(elems, op):
    # Section III-B taken literally: prefix scan of the reversed sequence with
    # the operator's operands left as they are.
    rev = L.all_prefix_sums(list(elems)[::-1], op)
    return rev[::-1]


CASES = {
    "combine_drop_C_eta": ("filter_combine", m_combine_drop_C_eta,
                           [lambda: P.test_lemma4_equals_definition1_joint(2),
                            lambda: P.test_parallel_formulation_equals_sequential("random")]),
    "combine_swapped_M": ("filter_combine", m_combine_swapped_M,
                          [lambda: P.test_lemma4_equals_definition1_joint(3),
                           lambda: P.test_parallel_formulation_equals_sequential("random")]),
    "combine_eta_sign": ("filter_combine", m_combine_eta_sign,
                         [lambda: P.test_lemma4_equals_definition1_joint(2),
                          lambda: P.test_lemma4_equals_definition1_quadrature()]),
    "combine_drop_Cj": ("filter_combine", m_combine_drop_Cj,
                        [lambda: P.test_lemma4_equals_definition1_quadrature(),
                         lambda: P.test_parallel_formulation_equals_sequential("tracking")]),
    "element_drop_F": ("filter_element", m_element_drop_F,
                       [lambda: P.test_lemma3_equals_joint_conditioning(3),
                        lambda: P.test_parallel_formulation_equals_sequential("random")]),
    "selem_drop_u": ("smoother_element", m_selem_drop_u,
                     [lambda: P.test_lemma5_equals_joint_conditioning(2),
                      lambda: P.test_parallel_formulation_equals_sequential("random")]),
    "selem_L_sign": ("smoother_element", m_selem_L_sign,
                     [lambda: P.test_lemma5_equals_joint_conditioning(4)]),
    "scomb_transpose": ("smoother_combine", m_scomb_transpose,
                        [lambda: P.test_lemma6_equals_definition2_monte_carlo(),
                         lambda: P.test_parallel_formulation_equals_sequential("random")]),
    "scomb_swap": ("smoother_combine", m_scomb_swap,
                   [lambda: P.test_lemma6_equals_definition2_quadrature(),
                    lambda: P.test_parallel_formulation_equals_sequential("tracking")]),
    "suffix_reversed_prefix": ("all_suffix_sums", m_suffix_reversed_prefix,
                               [lambda: P.test_suffix_sums_keep_left_operand_earlier(),
                                lambda: P.test_parallel_formulation_equals_sequential("tracking")]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, mutant, checks = CASES[name]
    monkeypatch.setattr(L, attr, mutant)
    for check in checks:
        with pytest.raises(AssertionError):
            check()


# ---------------------------------------------------------------- C oracle
# (original text, planted text, checks).  The mistake is planted in a copy of
# the C source compiled into a temporary directory.
C_CASES = {
    "kf_drop_Q": ("        for (int a = 0; a < n * n; ++a) Pp[a] += Qi[a];\n", "",
                  [lambda: P.test_kf_rts_equals_dense_posterior(3, 2, 6, False)]),
    "kf_drop_d": ("e[a] = y[i * m + a] - e[a] - di[a];", "e[a] = y[i * m + a] - e[a];",
                  [lambda: P.test_kf_rts_equals_dense_posterior(3, 2, 5, True)]),
    "rts_wrong_step_F": ("const double *Fk = F + (i + 1) * sF", "const double *Fk = F + i * sF",
                         [lambda: P.test_kf_rts_equals_dense_posterior(3, 2, 5, True)]),
    "rts_cov_sign": ("scov[i * n * n + a * n + c] = Pk[a * n + c] + s;",
                     "scov[i * n * n + a * n + c] = Pk[a * n + c] - s;",
                     [lambda: P.test_kf_rts_equals_dense_posterior(2, 1, 5, False),
                      lambda: P.test_scalar_random_walk_riccati(1.0, 1.0)]),
    "kf_gain_no_update": ("mk[a] = mp[a] + s;", "mk[a] = mp[a];",
                          [lambda: P.test_kf_rts_equals_dense_posterior(1, 1, 6, False)]),
}


@pytest.mark.parametrize("name", sorted(C_CASES))
def test_planted_c_mistake_is_caught(name, monkeypatch, tmp_path):
    orig, planted, checks = C_CASES[name]
    with open(os.path.join(os.path.dirname(oracle.__file__), "kf_rts.c")) as f:
        src = f.read()
    assert src.count(orig) >= 1, name
    mutant = os.path.join(tmp_path, "mutant.c")
    with open(mutant, "w") as f:
        f.write(src.replace(orig, planted, 1))
    so = os.path.join(tmp_path, "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", mutant, "-o", so, "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle.configure(ctypes.CDLL(so)))
    for check in checks:
        with pytest.raises(AssertionError):
            check()
