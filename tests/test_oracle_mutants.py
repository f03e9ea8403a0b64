"""The oracle's pins catch planted mistakes (CPU).

Each mutant is a copy of oracle/omp_oracle.c with one plausible mistake
planted by text replacement: a dropped term, a wrong sign, an off-by-one, a
wrong index or a transposed operand.  The copy is compiled to its own library
and the oracle pin tests (tests/test_oracle_*.py) run against it through the
OMPRT_ORACLE_LIB hook; at least one pin must fail.  A mutant that survives
names a reading of the paper that no pin holds the oracle to.  No mutant can
loop forever or read outside its arrays, and none is equivalent to the
original (a replacement that cannot change any result is left out).
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "omp_oracle.c")
PINS = [os.path.join(ROOT, "tests", f) for f in
        ("test_oracle_schedule.py", "test_oracle_bodies.py", "test_oracle_reduce.py",
         "test_oracle_misc.py")]

# (name, text in omp_oracle.c (exactly once), replacement)
MUTANTS = [
    # C0 trip count
    ("trip_count_off_by_one", "*n_out = q + 1;", "*n_out = q;"),
    ("trip_count_signedness",
     "empty = incr > 0 ? (ub < lb) : (ub > lb);",
     "empty = incr > 0 ? ((uint64_t)ub < (uint64_t)lb) : ((uint64_t)ub > (uint64_t)lb);"),
    ("widen_u32_sign_extends", "if (type == ORC_U32) return (int64_t)(uint32_t)v;",
     "if (type == ORC_U32) return (int64_t)(int32_t)v;"),
    ("incr_limit_unchecked",
     "if ((type == ORC_I32 || type == ORC_U32) && (incr > INT32_MAX || incr < -INT32_MAX))",
     "if (0 && (type == ORC_I32 || type == ORC_U32) && (incr > INT32_MAX || incr < -INT32_MAX))"),
    # C1 static without chunk
    ("static_start_index", "*start = k * q + (k < r ? k : r);", "*start = k * q + (k < r ? k : 0);"),
    ("static_count_drops_remainder", "*count = q + (k < r ? 1 : 0);", "*count = q;"),
    # C2 static chunk
    ("chunk_stride_drops_P", "*stride = orc_mul(P * c, incr);", "*stride = orc_mul(c, incr);"),
    ("chunk_last_owner", "*last = (nch > 0 && k == (nch - 1) % P);", "*last = (nch > 0 && k == nch % P);"),
    ("chunk_count_floor", "uint64_t nch = bn == 0 ? 0 : (bn - 1) / c + 1;",
     "uint64_t nch = bn == 0 ? 0 : bn / c;"),
    ("last_chunk_full_length", "cnt = (bn - s > c) ? c : bn - s;", "cnt = c;"),
    ("nochunk_stride", "*stride = orc_mul(bn, incr);", "*stride = orc_mul(bn - 1, incr);"),
    ("empty_piece_UB", "orc_add(*LB, -incr);", "orc_add(*LB, incr);"),
    # C3 composite table and owner maps
    ("composite_team_columns_swapped", "row[0] = tLB; row[1] = tUB; row[2] = tst; row[3] = tlast;",
     "row[0] = tUB; row[1] = tLB; row[2] = tst; row[3] = tlast;"),
    ("owner_map_chunk_end",
     "uint64_t a = j * chunk;\n                    uint64_t e = (bn - a > chunk) ? a + chunk : bn;",
     "uint64_t a = j * chunk;\n                    uint64_t e = (bn - a > chunk) ? a + chunk - 1 : bn;"),
    ("dist_chunk_end",
     "uint64_t a = k * chunk;\n                    uint64_t e = (bn - a > chunk) ? a + chunk : bn;",
     "uint64_t a = k * chunk;\n                    uint64_t e = (bn - a > chunk) ? a + chunk - 1 : bn;"),
    ("dist_team_of_chunk", "uint64_t g = j % G;", "uint64_t g = (j + 1) % G;"),
    # guided
    ("guided_divisor", "uint64_t want = (r + 2 * T - 1) / (2 * T);",
     "uint64_t want = (r + T - 1) / T;"),
    ("guided_skips_an_iteration", "next += size;", "next += size + 1;"),
    ("guided_min_chunk", "uint64_t size = want > c ? want : c;", "uint64_t size = want;"),
    # C6 bodies
    ("axpy_i32_transposed", "(uint32_t)alpha * (uint32_t)x[i] + (uint32_t)y[i]",
     "(uint32_t)alpha * (uint32_t)y[i] + (uint32_t)x[i]"),
    ("axpy_f32_transposed", "fmaf(alpha, x[i], y[i])", "fmaf(alpha, y[i], x[i])"),
    ("stencil1d_neighbour_index", "float nb = in[i - 1] + in[i + 1];", "float nb = in[i - 1] + in[i];"),
    ("stencil2d_sign", "float ew = in[i + 1] + in[i - 1];", "float ew = in[i + 1] - in[i - 1];"),
    ("stencil2d_coefficient_swap",
     "float ew = in[i + 1] + in[i - 1];\n                float ce = c0 * in[i];",
     "float ew = in[i + 1] + in[i - 1];\n                float ce = c1 * in[i];"),
    ("stencil2d_dropped_term", "out[i] = fmaf(c1, ns + ew, ce);", "out[i] = fmaf(c1, ns, ce);"),
    ("stencil2d_boundary_column", "if (r == 0 || c == 0 || r + 1 == ny || c + 1 == nx)",
     "if (r == 0 || c == 0 || r + 1 == ny)"),
    # C7 reductions
    ("sum_i32_zero_extends", "s += (uint64_t)(int64_t)a[i];", "s += (uint64_t)(uint32_t)a[i];"),
    ("max_f32_start", "double m = -INFINITY;", "double m = 0.0;"),
    ("min_i32_start",
     "int64_t orc_min_i32(uint64_t n, const int32_t *a)\n{\n    int64_t m = INT64_MAX;",
     "int64_t orc_min_i32(uint64_t n, const int32_t *a)\n{\n    int64_t m = 0;"),
    ("exact_round_ties_away",
     "if (rem > 0x400 || (rem == 0x400 && (sticky || (mant & 1)))) mant++;",
     "if (rem >= 0x400) mant++;"),
    ("exact_round_drops_sticky",
     "if (rem > 0x400 || (rem == 0x400 && (sticky || (mant & 1)))) mant++;",
     "if (rem > 0x400 || (rem == 0x400 && (mant & 1))) mant++;"),
    ("exact_carry_shift", "a->d[k] -= (int64_t)((uint64_t)c << 32);",
     "a->d[k] -= (int64_t)((uint64_t)c << 31);"),
    ("exact_add_high_digit_shift", "uint64_t hi = sh ? (m >> (64 - sh)) : 0;",
     "uint64_t hi = sh ? (m >> (63 - sh)) : 0;"),
    ("exact_add_sign_of_top_digit", "if (v < 0) { d0 = -d0; d1 = -d1; d2 = -d2; }",
     "if (v < 0) { d0 = -d0; d1 = -d1; }"),
    ("exact_round_drops_sign", "return neg ? -r : r;", "return r;"),
    ("plain_sum_fp32_accumulator", "double s = 0.0;\n    for (uint64_t i = 0; i < n; i++) s += (double)a[i];",
     "float s = 0.0f;\n    for (uint64_t i = 0; i < n; i++) s += a[i];"),
    ("plain_sum_right_to_left", "for (uint64_t i = 0; i < n; i++) s += (double)a[i];\n    return s;",
     "for (uint64_t i = n; i > 0; i--) s += (double)a[i - 1];\n    return s;"),
    ("plain_sum_drops_last", "for (uint64_t i = 0; i < n; i++) s += (double)a[i];\n    return s;",
     "for (uint64_t i = 0; i + 1 < n; i++) s += (double)a[i];\n    return s;"),
    ("exact_terms_first_only", "        kl_add(acc, -r);                        /* exact: r is a sum of addend bits */",
     "        return k;"),
    ("exact_terms_bf16_decode",
     "uint32_t bits = (uint32_t)a[i] << 16;\n        float f;\n        memcpy(&f, &bits, 4);\n        kl_add(&acc, (double)f);\n    }\n    return kl_terms",
     "uint32_t bits = (uint32_t)a[i] << 16;\n        float f;\n        memcpy(&f, &bits, 4);\n        kl_add(&acc, (double)f + 1.0);\n    }\n    return kl_terms"),
    ("abs_sum_without_abs", "kl_add(&acc, fabs((double)a[i]));", "kl_add(&acc, (double)a[i]);"),
    ("bf16_decode_shift",
     "double orc_exact_sum_bf16(uint64_t n, const uint16_t *a)\n{\n    orc_kulisch acc;\n    kl_init(&acc);\n    for (uint64_t i = 0; i < n; i++) {\n        uint32_t bits = (uint32_t)a[i] << 16;",
     "double orc_exact_sum_bf16(uint64_t n, const uint16_t *a)\n{\n    orc_kulisch acc;\n    kl_init(&acc);\n    for (uint64_t i = 0; i < n; i++) {\n        uint32_t bits = (uint32_t)a[i] << 15;"),
    ("dot_transposed_operand", "kl_add(&acc, (double)x[i] * (double)y[i]);",
     "kl_add(&acc, (double)x[i] * (double)x[i]);"),
    # C8 atomic inc
    ("atomic_inc_wrap", "*x = (v >= e) ? 0u : v + 1u;", "*x = (v > e) ? 0u : v + 1u;"),
    # C10 stack
    ("stack_zero_size_request", "uint64_t r = ((b == 0 ? 1 : b) + 15) / 16 * 16;",
     "uint64_t r = (b + 15) / 16 * 16;"),
    ("stack_free_order_unchecked", "if (region == 0 && off + r == top_s) top_s = off;",
     "if (region == 0) top_s = off;"),
    ("stack_nomem_bit_dropped", "region = 2; status |= ORC_STACK_NOMEM;", "region = 2;"),
    ("stack_free_of_failed_alloc_flagged", "else if (region == 2) bits = 0;",
     "else if (region == 2) bits = ORC_STACK_ORDER;"),
    ("stack_pool_capacity", "} else if (r <= Q - top_q && top_q <= Q) {",
     "} else if (r <= Q && top_q <= Q) {"),
    # C12 MLP and Adam
    ("mlp_relu_dropped", "out[o] = (relu && s < 0.0) ? 0.0 : s;", "out[o] = s;"),
    ("mlp_output_layer_relu",
     "mlp_layer(p + OFF_W3, p + OFF_B3, h2, M_H, M_OUT, 0, Y + r * M_OUT);",
     "mlp_layer(p + OFF_W3, p + OFF_B3, h2, M_H, M_OUT, 1, Y + r * M_OUT);"),
    ("mlp_grad_w2_transposed", "grad[OFF_W2 + o * M_H + i] += dh2[o] * h1[i];",
     "grad[OFF_W2 + i * M_H + o] += dh2[o] * h1[i];"),
    ("mlp_backprop_relu_gate", "dh1[i] = h1[i] > 0.0 ? s : 0.0;", "dh1[i] = s;"),
    ("mlp_loss_grad_factor", "dy[o] = 2.0 * d * scale;", "dy[o] = d * scale;"),
    ("adam_second_moment_not_squared", "v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];",
     "v[i] = b2 * v[i] + (1.0 - b2) * g[i];"),
    ("adam_bias_correction", "double mh = m[i] / c1, vh = v[i] / c2;",
     "double mh = m[i], vh = v[i] / c2;"),
]


def _run_mutant(m, workdir):
    name, old, new = m
    src = open(SRC).read()
    assert src.count(old) == 1, "%s: the planted text must occur exactly once" % name
    c = os.path.join(workdir, name + ".c")
    so = os.path.join(workdir, name + ".so")
    with open(c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-w", "-o", so, c, "-lm"])
    env = dict(os.environ, OMPRT_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"] + PINS, cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-200:]
    return name, r.returncode, tail


def test_every_planted_mistake_fails_a_pin():
    if os.environ.get("OMPRT_ORACLE_LIB"):
        pytest.skip("already running against a mutant")
    with tempfile.TemporaryDirectory() as d:
        with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda m: _run_mutant(m, d), MUTANTS))
    survived = [(n, tail) for n, rc, tail in results if rc == 0]
    assert not survived, "mutants no pin catches: %s" % survived


def test_unmutated_copy_passes_the_pins():
    """The harness itself: the same compile-and-run path with no mistake
    planted passes every pin (so a caught mutant is caught by its mistake)."""
    if os.environ.get("OMPRT_ORACLE_LIB"):
        pytest.skip("already running against a mutant")
    with tempfile.TemporaryDirectory() as d:
        name, rc, tail = _run_mutant(("unmutated", "*n_out = q + 1;", "*n_out = q + 1;"), d)
    assert rc == 0, tail
