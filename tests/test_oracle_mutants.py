"""Do the oracle's pins catch plausible mistakes?  (CPU only.)

Each case compiles a copy of oracle/fmm_oracle.c with ONE mistake planted -- a
flipped sign, a power or index off by one, a transposed or conjugated operand, a
wrong binomial, a dropped factor, a wrong neighbourhood test -- points the
oracle's Python wrapper at that copy, and runs the pins that guard the part it
touched (Eq. M2Lmat; the interaction lists of Sec. 4.1; the P2M / M2M of
Sec. 2.1; the Hermite functions and Eq. C_beta; Eq. n_body over adjacent boxes).
At least one of them must fail.  The unmodified copy, built the same way,
passes all of them.  Nothing here touches the GPU or the CUDA library.  Every
planted mistake keeps the oracle's memory accesses in bounds (a list test that
let adjacent boxes in would overrun the 27-entry list buffers and end the
process, not fail a pin).
"""
import contextlib
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_adaptive as ta
import test_oracle_fgt as tf
import test_oracle_m2l as tm
import test_oracle_nearfield as tn
import workloads

SRC = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "fmm_oracle.c")


def _pts():
    return workloads.uniform_particles(800, np.random.default_rng(71))


# the pins guarding each part of the oracle (pytest functions called with explicit arguments)
PINS = {
    "m2l": [
        lambda o: tm.test_m2l_point_source_at_centre_is_exact_taylor(o),
        lambda o: tm.test_m2l_converges_to_exact_taylor_coefficients(o),
        lambda o: tm.test_m2m_then_m2l_equals_parent_p2m(o),
    ],
    "lists": [
        lambda o: tm.test_list_matches_all_pairs_brute_force(o, 3),
        lambda o: tm.test_list_count_closed_form(o, 4),
    ],
    "upward": [
        lambda o: tm.test_m2m_then_m2l_equals_parent_p2m(o),
        lambda o: tn.test_whole_fmm_converges_to_the_direct_sum(o, _pts(), 3),
    ],
    "fgt": [
        lambda o: tf.test_hermite_functions_match_numpy(o),
        lambda o: tf.test_h2t_of_single_source_equals_its_taylor_coefficients(o),
        lambda o: tf.test_h2t_separable_hankel_form(o),
    ],
    "near": [
        lambda o: tn.test_near_field_skips_only_the_coincident_source(o, _pts()),
        lambda o: tn.test_near_field_is_the_sum_over_adjacent_boxes(o, _pts(), 3),
    ],
    "adjoint": [
        lambda o: tm.test_adjoint_dot_product(o, False),
        lambda o: tm.test_operator_transpose_identity(o),
    ],
    "farfield": [
        lambda o: tm.test_m2p_centred_source_is_exact(o),
        lambda o: tm.test_m2p_single_term_powers(o),
        lambda o: tm.test_m2p_equals_l2p_of_m2l_in_the_limit(o),
        lambda o: tm.test_far_field_potential_converges_geometrically(o, tm.small_tree_case()),
        lambda o: tn.test_whole_fmm_converges_to_the_direct_sum(o, _pts(), 3),
    ],
    "adaptive": [
        lambda o: ta.test_tree_matches_recursive_builder(o, ta.small_case(o)),
        lambda o: ta.test_tree_invariants(o, ta.small_case(o)),
        lambda o: ta.test_vlists_brute_force_and_symmetric(o, ta.small_case(o)),
    ],
    "fgt_expansions": [
        lambda o: tf.test_hermite_expansion_converges_to_direct(o, tf.fgt_case()),
        lambda o: tf.test_taylor_expansion_converges_to_direct(o, tf.fgt_case()),
        lambda o: tf.test_full_fgt_grid_pipeline_matches_direct(o),
        lambda o: tf.test_hermite_grid_eval_sums_exactly_the_neighbourhood(o, 2),
    ],
}

# (name, guarded part, text in fmm_oracle.c, the same text with the mistake planted)
MUTANTS = [
    ("m2l_sign_flipped", "m2l",
     "cplx a = sign * binom(n + k, k) * pw[n + k + 1];",
     "cplx a = -sign * binom(n + k, k) * pw[n + k + 1];"),
    ("m2l_power_off_by_one", "m2l",
     "cplx a = sign * binom(n + k, k) * pw[n + k + 1];",
     "cplx a = sign * binom(n + k, k) * pw[n + k];"),
    ("m2l_wrong_binomial", "m2l",
     "cplx a = sign * binom(n + k, k) * pw[n + k + 1];",
     "cplx a = sign * binom(n + k + 1, k) * pw[n + k + 1];"),
    ("m2l_conjugated_me", "m2l",
     "s += a * (m[2 * k] + I * m[2 * k + 1]);",
     "s += a * (m[2 * k] - I * m[2 * k + 1]);"),
    ("m2l_transposed_index", "m2l",
     "s += a * (m[2 * k] + I * m[2 * k + 1]);",
     "s += a * (m[2 * n] + I * m[2 * n + 1]);"),
    ("lists_separation_too_strict", "lists",
     "if (cheb < 2) continue; /* adjacent (or itself): near field */",
     "if (cheb < 3) continue; /* adjacent (or itself): near field */"),
    ("m2m_shift_reversed", "upward",
     "cplx z = box_centre(child_level, ix, iy) - box_centre(child_level - 1, ix >> 1, iy >> 1);",
     "cplx z = box_centre(child_level - 1, ix >> 1, iy >> 1) - box_centre(child_level, ix, iy);"),
    ("m2m_power_index", "upward",
     "for (int k = 0; k <= j; ++k) s += binom(j, k) * zp[j - k] * (mc[2 * k] + I * mc[2 * k + 1]);",
     "for (int k = 0; k <= j; ++k) s += binom(j, k) * zp[k] * (mc[2 * k] + I * mc[2 * k + 1]);"),
    ("p2m_power_off_by_one", "upward",
     "cplx t = c[i] * pw;",
     "cplx t = c[i] * pw * d;"),
    ("hermite_recurrence_coefficient", "fgt",
     "h[n + 1] = 2.0 * t * h[n] - 2.0 * (double)n * h[n - 1];",
     "h[n + 1] = 2.0 * t * h[n] - 2.0 * (double)(n + 1) * h[n - 1];"),
    ("h2t_sign_dropped", "fgt",
     "double sign = ((b1 + b2) % 2 == 0) ? 1.0 : -1.0;\n            C[b1 * p + b2] += sign",
     "double sign = 1.0;\n            C[b1 * p + b2] += sign"),
    ("h2t_transposed_hankel", "fgt",
     "s += A[a1 * p + a2] * h1[a1 + b1] * h2[a2 + b2];",
     "s += A[a1 * p + a2] * h1[a1 + b2] * h2[a2 + b1];"),
    ("near_field_cross_not_square", "near",
     "if (abs(sx - tx) > 1 || abs(sy - ty) > 1) continue;",
     "if (abs(sx - tx) > 1 && abs(sy - ty) > 1) continue;"),
    ("near_field_self_not_skipped", "near",
     "if (xy[2 * i] == z[2 * j] && xy[2 * i + 1] == z[2 * j + 1]) continue;",
     ";"),
    ("adjoint_not_transposed", "adjoint",
     "cplx anks = a[2 * (nn * p + k)] + I * a[2 * (nn * p + k) + 1];",
     "cplx anks = a[2 * (k * p + nn)] + I * a[2 * (k * p + nn) + 1];"),
    ("l2l_power_index", "farfield",
     "for (int n = j; n < p; ++n) s += binom(n, j) * zp[n - j] * (lp[2 * n] + I * lp[2 * n + 1]);",
     "for (int n = j; n < p; ++n) s += binom(n, j) * zp[j] * (lp[2 * n] + I * lp[2 * n + 1]);"),
    ("l2p_power_off_by_one", "farfield",
     "cplx s = 0.0, pw = 1.0;",
     "cplx s = 0.0, pw = w;"),
    ("m2p_power_off_by_one", "farfield",
     "cplx s = 0.0, pw = 1.0 / w;",
     "cplx s = 0.0, pw = 1.0;"),
    ("adaptive_split_at_q", "adaptive",
     "int parent_split = exists[level_offset(l - 1) + pb] && cnt_parent[pb] > q;",
     "int parent_split = exists[level_offset(l - 1) + pb] && cnt_parent[pb] >= q;"),
    ("vlist_separation_too_strict", "adaptive",
     "if ((adx > ady ? adx : ady) <= 1) continue; /* adjacent: U-list, near field */",
     "if ((adx > ady ? adx : ady) <= 2) continue; /* adjacent: U-list, near field */"),
    ("p2h_factorials_dropped", "fgt_expansions",
     "A[a1 * p + a2] += q[j] * w1[a1] * w2[a2] / (f[a1] * f[a2]);",
     "A[a1 * p + a2] += q[j] * w1[a1] * w2[a2];"),
    ("taylor_power_off_by_one", "fgt_expansions",
     "s += B[b1 * p + b2] * pow(t1, b1) * pow(t2, b2);",
     "s += B[b1 * p + b2] * pow(t1, b1 + 1) * pow(t2, b2);"),
    ("p2h_grid_box_corner_not_centre", "fgt_expansions",
     "double t1 = (x[2 * j] - ((double)ix + 0.5) * side) / sc;",
     "double t1 = (x[2 * j] - ((double)ix) * side) / sc;"),
    ("hermite_grid_neighbourhood_short", "fgt_expansions",
     "double acc = 0.0;\n        for (int sy = ty - ncut; sy <= ty + ncut; ++sy) {",
     "double acc = 0.0;\n        for (int sy = ty - ncut; sy < ty + ncut; ++sy) {"),
]


def _compile(src_text: str, path: str) -> str:
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", path, c, "-lm"])
    return path


@contextlib.contextmanager
def _oracle_from(path: str):
    """The oracle's Python wrapper, calling into the library at `path` for the duration."""
    lib = ctypes.CDLL(path)
    for name, (res, args) in oracle._SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    oracle.lib()  # the real library is loaded first, so it is what is restored
    saved = oracle._lib
    oracle._lib = lib
    try:
        yield oracle
    finally:
        oracle._lib = saved


def _failures(o, part: str):
    failed = []
    for i, pin in enumerate(PINS[part]):
        try:
            with np.errstate(all="ignore"):
                pin(o)
        except AssertionError:
            failed.append(i)
    return failed


@pytest.fixture(scope="module")
def src_text():
    with open(SRC) as f:
        return f.read()


def test_unmodified_copy_passes_every_pin(tmp_path_factory, src_text):
    path = _compile(src_text, str(tmp_path_factory.mktemp("oracle_copy") / "liborc_copy.so"))
    with _oracle_from(path) as o:
        for part in PINS:
            assert _failures(o, part) == [], part


@pytest.mark.parametrize("name,part,orig,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path_factory, src_text, name, part, orig, planted):
    assert src_text.count(orig) == 1, "the mutation site must be unique in fmm_oracle.c"
    path = _compile(src_text.replace(orig, planted), str(tmp_path_factory.mktemp(name) / f"liborc_{name}.so"))
    with _oracle_from(path) as o:
        assert _failures(o, part), f"no pin of '{part}' caught the planted mistake {name}"
