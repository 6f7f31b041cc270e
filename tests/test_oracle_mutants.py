"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a private copy of ``oracle/pano_oracle.c``
(a flipped sign, a swapped operand, a dropped term ...), compiles it on the
CPU, points the oracle front end at the mutant and runs the pins of
``test_oracle_pins``. At least one pin must fail for every mutant. The real
oracle is restored afterwards.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_compose_pins as cpins
from tests import test_oracle_pins as pins
from tests import test_oracle_refine_pins as rpins
from tests import test_oracle_storage_pins as spins

SRC = os.path.join(os.path.dirname(oracle.__file__), "pano_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("It sign", "- T[q];\n            s[q]", "+ T[q];\n            s[q]"),
    ("s uses Iy for x", "s[q] = Ix[q] * u[2 * q] + Iy[q]", "s[q] = Iy[q] * u[2 * q] + Iy[q]"),
    ("s drops linearisation", "s[q] = Ix[q] * u[2 * q] + Iy[q] * u[2 * q + 1] - It;", "s[q] = -It;"),
    ("damping term dropped", "double r1 = m1 + lambda * u[2 * p]", "double r1 = m1 + 0.0 * u[2 * p]"),
    ("solve transposed", "v[2 * p + 0] = (a22 * r1 - g12 * r2) / det;", "v[2 * p + 0] = (a11 * r1 - g12 * r2) / det;"),
    ("window clamped not clipped", "if (qx < 0 || qx >= w) continue;", "if (0) continue;"),
    ("upsample not doubled", "uf[2 * p + 0] = 2.0 *", "uf[2 * p + 0] = 1.0 *"),
    ("upsample wrong scale", "0.5 * x, 0.5 * y);\n            uf[2 * p + 1]", "0.5 * x, 0.5 * x);\n            uf[2 * p + 1]"),
    ("pyramid odd kernel", "{1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};\n    int hd = (h + 1) / 2, wd = (w + 1) / 2;\n    double* tmp",
     "{1.0 / 16, 4.0 / 16, 6.0 / 16, 5.0 / 16, 0.0 / 16};\n    int hd = (h + 1) / 2, wd = (w + 1) / 2;\n    double* tmp"),
    ("pyramid keeps odd rows", "int y = 2 * yd, x = 2 * xd;", "int y = 2 * yd + 1, x = 2 * xd;"),
    ("bilinear fx/fy swapped", "return (1.0 - fy) * ((1.0 - fx) * i00 + fx * i10) + fy * ((1.0 - fx) * i01 + fx * i11);\n}\n\ndouble oracle_bilinear(",
     "return (1.0 - fx) * ((1.0 - fy) * i00 + fy * i10) + fy * ((1.0 - fx) * i01 + fx * i11);\n}\n\ndouble oracle_bilinear("),
    ("gradient halved twice", "PIX(Ix, w, y, x) = 0.5 *", "PIX(Ix, w, y, x) = 0.25 *"),
    ("luma weights", "0.299 * img[3 * i + 0] + 0.587", "0.587 * img[3 * i + 0] + 0.299"),
    ("blend position uses BlendL", "double Lx = x + rlx * (1.0 - blendL)", "double Lx = x + rlx * blendL"),
    ("blend flow roles swapped", "double Rx = x + lrx * (1.0 - blendR)", "double Rx = x + rlx * (1.0 - blendR)"),
    ("FlowMag roles swapped", "double expL = exp(k_sharp * blendL * (1.0 + k_mag * magRL));",
     "double expL = exp(k_sharp * blendL * (1.0 + k_mag * magLR));"),
    ("softmax sign", "double expR = exp(k_sharp * blendR", "double expR = exp(-k_sharp * blendR"),
    ("Eq1 ramp off by one", "out[x] = (double)(x + 1) / (double)(w + 1);", "out[x] = (double)(x) / (double)(w + 1);"),
    ("Eq1 distance squared", "double d = sqrt(", "double d = ("),
    ("quantize truncates", "double v = nearbyint(255.0 * F[i]);", "double v = floor(255.0 * F[i]);"),
    ("energy smoothness one-sided", "if (y < h - 1) { double d = u[2 * (p + w) + c] - u[2 * p + c]; smooth += d * d; }",
     "if (0) { double d = 0; smooth += d * d; }"),
    ("energy grad drops factor 2", "gu[2 * p + c] += 2.0 * alpha * s;", "gu[2 * p + c] += alpha * s;"),
    ("energy grad T sign", "if (gT) gT[p] = -2.0 * r;", "if (gT) gT[p] = 2.0 * r;"),
    ("energy grad J tap weight", "PIX(gJ, w, ya, xb) += g * (1.0 - fy) * fx;", "PIX(gJ, w, ya, xb) += g * fy * fx;"),
    ("energy grad derivative axis", "*dx = (1.0 - fy) * (i10 - i00) + fy * (i11 - i01);",
     "*dx = (1.0 - fx) * (i10 - i00) + fx * (i11 - i01);"),
    ("bfloat16 significand bits", "int p = fmt == 1 ? 8 : 11;", "int p = fmt == 1 ? 9 : 11;"),
    ("storage rounds down", "double r = nearbyint(v / ulp) * ulp;", "double r = floor(v / ulp) * ulp;"),
    ("storage without subnormal spacing", "if (lead < emin) lead = emin;", "if (0) lead = emin;"),
    ("stored level not rounded", "        oracle_round_storage(cur, (long)hs[l] * ws[l], fmt);\n", "\n"),
    ("reduce adjoint weight", "PIX(gsrc, w, sy, sx) += k[ty + 2] * k[tx + 2] * g;",
     "PIX(gsrc, w, sy, sx) += k[ty + 2] * k[ty + 2] * g;"),
    ("compose Area1 copies R", "/* Code 1: F(i, j) = L(i, j) */\n                for (int ch = 0; ch < c; ++ch) out[ch] = L[p * c + ch];",
     "/* Code 1: F(i, j) = L(i, j) */\n                for (int ch = 0; ch < c; ++ch) out[ch] = R[p * c + ch];"),
    ("compose crop origin sign", "int qy = y - fy0, qx = x - fx0;", "int qy = y + fy0, qx = x - fx0;"),
    ("compose ColorR with FlowRtoL", "double Rx_ = x + (1.0 - BlendR) * ltor_x", "double Rx_ = x + (1.0 - BlendR) * rtol_x"),
    ("compose FlowMag over canvas width", "double FlowMagRL = sqrt(rtol_x * rtol_x + rtol_y * rtol_y) / (double)fw;",
     "double FlowMagRL = sqrt(rtol_x * rtol_x + rtol_y * rtol_y) / (double)w;"),
    ("compose neither not zero", "/* Code 1: F(i, j) = 0 */\n                for (int ch = 0; ch < c; ++ch) out[ch] = 0.0;",
     "/* Code 1: F(i, j) = 0 */\n                for (int ch = 0; ch < c; ++ch) out[ch] = 0.5;"),
]

PIN_TESTS = [
    lambda: pins.test_luma_gray_is_identity_and_weights_are_bt601(),
    lambda: [pins.test_pyr_down_matches_scipy_binomial_reduce(s) for s in [(7, 9), (8, 8)]],
    lambda: pins.test_bilinear_matches_scipy_order1_nearest(),
    lambda: pins.test_gradient_is_central_difference_with_replicate_border(),
    lambda: [pins.test_lk_step_matches_bruteforce_least_squares(r, l) for r, l in [(1, 1e-3), (2, 1e-2)]],
    lambda: pins.test_lk_step_integer_translation_is_a_fixed_point_and_attracts(),
    lambda: pins.test_upsample_flow_matches_scipy_and_doubles(),
    lambda: pins.test_flow_pair_recovers_subpixel_translation(),
    lambda: pins.test_flow_pair_needs_the_pyramid_for_large_motion(),
    lambda: [pins.test_blend_coeff_golden_eq1(c) for c in pins._read_golden_canvases()],
    lambda: [pins.test_blend_ramp_is_eq1_for_a_strip(w) for w in (4, 9)],
    lambda: [pins.test_blend_closed_form_for_constant_translation(d) for d in [(2.0, -1.0)]],
    lambda: pins.test_blend_swap_symmetry_exact(),
    lambda: pins.test_blend_mirror_symmetry_with_strip_ramp(),
    lambda: pins.test_blend_weights_sum_to_one_and_follow_the_blend_coefficient(),
    lambda: pins.test_blend_larger_RtoL_flow_pulls_weight_towards_L(),
    lambda: pins.test_quantize_u8_rounds_half_to_even_and_clamps(),
    lambda: [rpins.test_energy_gradient_in_u_matches_central_differences(a) for a in (0.0, 0.05)],
    lambda: rpins.test_energy_gradients_in_T_and_J_match_central_differences(),
    lambda: rpins.test_smoothness_energy_closed_form(),
    lambda: rpins.test_energy_and_gradients_vanish_on_identical_images_and_zero_flow(),
    lambda: [rpins.test_reduce_transpose_dot_product_identity(s) for s in [(7, 9), (13, 2)]],
    lambda: cpins.test_area1_area2_and_neither_are_copies_and_zeros(),
    lambda: [cpins.test_area3_constant_translation_closed_form(d) for d in [(2, -1)]],
    lambda: cpins.test_swapping_the_roles_of_L_and_R_is_exact(),
    lambda: cpins.test_crop_origin_places_the_flows_on_the_canvas(),
    lambda: cpins.test_strip_canvas_reduces_to_the_strip_form(),
    lambda: spins.test_binary16_rounding_matches_numpy(),
    lambda: spins.test_bfloat16_rounding_matches_torch_on_float32_inputs(),
    lambda: spins.test_ties_go_to_the_even_neighbour(),
    lambda: [spins.test_stored_pyramid_is_representable_and_close_to_the_exact_one(f, p)
             for f, p in [(oracle.FMT_BF16, 8), (oracle.FMT_F16, 11)]],
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not unique in the oracle source"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", str(mpath), "-o", str(so), "-lm"])
    return str(so)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, name, old, new):
    so = _build_mutant(tmp_path, name, old, new)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: so)
    caught = []
    try:
        for i, t in enumerate(PIN_TESTS):
            try:
                t()
            except AssertionError:
                caught.append(i)
    finally:
        oracle._lib = None
    assert caught, f"no pin caught the planted mistake {name!r}"
