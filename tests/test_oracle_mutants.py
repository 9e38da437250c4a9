"""Planted mistakes: each mutant below is a copy of oracle/chp.c with one
plausible slip (a dropped term, a wrong sign, index, branch or operand),
built with gcc; the oracle pins (tests/test_oracle.py) must fail on every
mutant and pass on the unmodified oracle.  Each pin run is a child process
pointed at its library through ORACLE_LIB, so a mutant that corrupts memory
ends only that process.  CPU only."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "chp.c")

# name -> (text in chp.c, replacement); each text occurs exactly once
MUTANTS = {
    # Sec. 2.4 gate table
    "cx_phase_as_printed": ("s->r[i] ^= (uint8_t)(xa & zb & (xb ^ za ^ 1));",
                            "s->r[i] ^= (uint8_t)(xa & zb);"),
    "cx_target_z": ("setb(z, a, za ^ zb);\n            break;\n        case K_CZ:",
                    "setb(z, b, za ^ zb);\n            break;\n        case K_CZ:"),
    "cz_rule": ("setb(z, a, za ^ xb);", "setb(z, a, za ^ zb);"),
    "h_sign_dropped": ("s->r[i] ^= (uint8_t)(xa & za);\n            setb(x, a, za); setb(z, a, xa);",
                       "setb(x, a, za); setb(z, a, xa);"),
    "s_sign_from_post_gate_bits": ("s->r[i] ^= (uint8_t)(xa & za);\n            setb(z, a, za ^ xa);",
                                   "setb(z, a, za ^ xa);\n            s->r[i] ^= (uint8_t)(xa & (za ^ xa));"),
    "y_sign": ("case K_Y: s->r[i] ^= (uint8_t)(xa ^ za); break;",
               "case K_Y: s->r[i] ^= (uint8_t)(xa & za); break;"),
    "swap_one_plane": ("setb(z, a, zb); setb(z, b, za);", "setb(z, a, za); setb(z, b, zb);"),
    # Appendix B: g and rowsum
    "g_sign_y": ("if (x1 == 1 && z1 == 1) return z2 - x2;", "if (x1 == 1 && z1 == 1) return x2 - z2;"),
    "g_x_branch": ("return z2 * (2 * x2 - 1);", "return z2 * (1 - 2 * x2);"),
    "rowsum_sign_term_dropped": ("long long sum = 2 * (long long)s->r[h] + 2 * (long long)s->r[i];",
                                 "long long sum = 2 * (long long)s->r[h];"),
    "rowsum_branch_swapped": ("if (m == 0) s->r[h] = 0;\n    else if (m == 2) s->r[h] = 1;",
                              "if (m == 0) s->r[h] = 1;\n    else if (m == 2) s->r[h] = 0;"),
    # (swapping the two rows' roles in g is no mistake: CHP multiplies only
    # commuting rows, whose product has the same power of i in either order,
    # apart from the pivot's destabilizer partner, which is overwritten next)
    "rowsum_x_z_transposed": ("sum += chp_g(bit(xi, j), bit(zi, j), bit(xh, j), bit(zh, j));",
                              "sum += chp_g(bit(xi, j), bit(zi, j), bit(zh, j), bit(xh, j));"),
    # Sec. 2.4 measurement
    "pivot_skips_first_stabilizer": ("for (uint32_t i = n; i < 2 * n; i++)\n        if (bit(XR(s, i), a))",
                                     "for (uint32_t i = n + 1; i < 2 * n; i++)\n        if (bit(XR(s, i), a))"),
    "destabilizer_sign_not_copied": ("s->r[p - n] = s->r[p];\n        memset(XR(s, p), 0",
                                     "s->r[p - n] = 0;\n        memset(XR(s, p), 0"),
    "outcome_sign_inverted": ("setb(ZR(s, p), a, 1);\n        s->r[p] = (uint8_t)(coin & 1);",
                              "setb(ZR(s, p), a, 1);\n        s->r[p] = (uint8_t)(1 - (coin & 1));"),
    "deterministic_uses_destabilizers": ("int m = rowsum(s, sc, i + n);\n        cntK++;\n        if (m & 1) return OR_ODD_PHASE;\n    }\n    /* The",
                                         "int m = rowsum(s, sc, i);\n        cntK++;\n        if (m & 1) return OR_ODD_PHASE;\n    }\n    /* The"),
    "reset_flip_skipped": ("} else if (out) {\n                apply_pauli(s, a, 1);",
                           "} else if (0) {\n                apply_pauli(s, a, 1);"),
    # Sec. 3.2 commutation and Pauli-product measurement
    "commute_term_dropped": ("acc += bit(xp, j) * bit(zs, j) + bit(zp, j) * bit(xs, j);",
                             "acc += bit(xp, j) * bit(zs, j);"),
    "mpp_destabilizer_sign_not_copied": ("s->r[p - n] = s->r[p];\n        memcpy(XR(s, p), XR(s, pr)",
                                         "s->r[p - n] = 0;\n        memcpy(XR(s, p), XR(s, pr)"),
    "mpp_y_factor_without_z": ("if (c == 2 || c == 3) setb(ZR(s, pr), q, 1);",
                               "if (c == 3) setb(ZR(s, pr), q, 1);"),
    # Sec. 2.7 noise channels, Sec. 4.2 composite channel
    "threshold_off_by_one": ("return (uint64_t)(p * 4294967296.0);", "return (uint64_t)(p * 4294967296.0) + 1;"),
    "dep1_pauli_order": ("apply_pauli(s, a, (int)((u * 3) / T) + 1);", "apply_pauli(s, a, 3 - (int)((u * 3) / T));"),
    "dep2_qubits_swapped": ("if (m / 4) apply_pauli(s, a, m / 4);\n                        if (m % 4) apply_pauli(s, b, m % 4);",
                            "if (m % 4) apply_pauli(s, a, m % 4);\n                        if (m / 4) apply_pauli(s, b, m / 4);"),
    "pc1_y_as_z": ("else if (u < tx + ty) P = 2;", "else if (u < tx + ty) P = 3;"),
    "reset_error_phase_as_x": ("if (u2 < thr(pp[1])) { apply_pauli(s, a, 3);", "if (u2 < thr(pp[1])) { apply_pauli(s, a, 1);"),
    "reset_error_coin_bit": ("int out = measure(s, a, (int)(u1 & 1u), st);", "int out = measure(s, a, (int)((u1 >> 1) & 1u), st);"),
}


def _build(src_text, path):
    with open(path + ".c", "w") as fh:
        fh.write(src_text)
    r = subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", path + ".c", "-o", path],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return path


def _pins_pass(lib_path):
    env = dict(os.environ, ORACLE_LIB=lib_path)
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle.py", "-x", "-q",
                            "-p", "no:cacheprovider", "-m", "not gpu"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return False, "timeout"
    return r.returncode == 0, (r.stdout + r.stderr)[-600:]


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    out = {"original": _build(src, str(d / "liboriginal.so"))}
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, f"{name}: the mutated text must occur exactly once in chp.c"
        out[name] = _build(src.replace(old, new), str(d / f"lib{name}.so"))
    return out


def test_every_planted_mistake_fails_a_pin_and_the_oracle_passes(libs):
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        res = dict(zip(libs, ex.map(_pins_pass, libs.values())))
    ok, log = res.pop("original")
    assert ok, "the unmodified oracle fails its pins:\n" + log
    survivors = [name for name, (passed, _) in res.items() if passed]
    assert not survivors, f"mistakes no pin catches: {survivors}"
