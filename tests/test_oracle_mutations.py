"""The oracle's pins catch planted mistakes.  Each mutant is a copy of
oracle/qsim_oracle.c with one plausible error (a flipped sign, a dropped
factor or conjugate, a transposed operand, a wrong index or bit order, a lost
control), compiled on the CPU like the oracle itself and loaded by the pin
files (tests/test_oracle_pins.py, tests/test_mmd_pins.py) in a process of its
own; every mutant must fail at least one pin, and the unmodified source
compiled the same way must pass them all."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qsim_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_mmd_pins.py"]

# name: (text in qsim_oracle.c, replacement)
MUTANTS = {
    "rx_sign": ("U[0] = c; U[1] = -I * s; U[2] = -I * s; U[3] = c;", "U[0] = c; U[1] = I * s; U[2] = I * s; U[3] = c;"),
    "ry_transposed": ("U[0] = c; U[1] = -s; U[2] = s; U[3] = c;", "U[0] = c; U[1] = s; U[2] = -s; U[3] = c;"),
    "rz_half_angle_dropped": ("U[0] = cexp(-I * theta / 2); U[3] = cexp(I * theta / 2);",
                              "U[0] = cexp(-I * theta); U[3] = cexp(I * theta);"),
    "t_is_s": ("case ORC_T: U[0] = 1; U[3] = cexp(I * M_PI / 4);", "case ORC_T: U[0] = 1; U[3] = cexp(I * M_PI / 2);"),
    "shift_on_zero": ("case ORC_SHIFT: U[0] = 1; U[3] = cexp(I * theta);", "case ORC_SHIFT: U[0] = cexp(I * theta); U[3] = 1;"),
    "swap_is_identity": ("U[0 * 4 + 0] = 1; U[1 * 4 + 2] = 1; U[2 * 4 + 1] = 1; U[3 * 4 + 3] = 1;",
                         "U[0 * 4 + 0] = 1; U[1 * 4 + 1] = 1; U[2 * 4 + 2] = 1; U[3 * 4 + 3] = 1;"),
    "rot_sign": ("U[r * K + col] = (r == col ? c : 0) - I * s * prod;", "U[r * K + col] = (r == col ? c : 0) + I * s * prod;"),
    "pauli_y_transposed": ("if (p == 2) { m[0][1] = -I; m[1][0] = I; }", "if (p == 2) { m[0][1] = I; m[1][0] = -I; }"),
    "controls_inverted": ("if ((((uint64_t)b >> ctrl_locs[c]) & 1u) != (uint64_t)ctrl_vals[c]) match = 0;",
                          "if ((((uint64_t)b >> ctrl_locs[c]) & 1u) == (uint64_t)ctrl_vals[c]) match = 0;"),
    "matrix_transposed": ("for (int mm = 0; mm < K; ++mm) acc += U[m * K + mm] * x[mm];",
                          "for (int mm = 0; mm < K; ++mm) acc += U[mm * K + m] * x[mm];"),
    "target_bits_reversed": ("if ((m >> j) & 1) i |= 1ull << locs[j];", "if ((m >> j) & 1) i |= 1ull << locs[k - 1 - j];"),
    "dagger_without_transpose": ("for (int col = 0; col < K; ++col) U[r * K + col] = conj(M[col * K + r]);",
                                 "for (int col = 0; col < K; ++col) U[r * K + col] = conj(M[r * K + col]);"),
    "dagger_keeps_s": ("case ORC_S: d.kind = ORC_SDG; return", "case ORC_S: d.kind = ORC_S; return"),
    "dagger_keeps_angle": ("return orc_gate_matrix(&d, -theta, mats, U);", "return orc_gate_matrix(&d, theta, mats, U);"),
    "expect_without_conj": ("prod[i] = creal(conj(psi[i]) * phi[i]);", "prod[i] = creal(psi[i] * phi[i]);"),
    "expect_drops_coeff": ("vals[t] = terms[t].coeff * orc_pairwise_sum(prod, dim);", "vals[t] = orc_pairwise_sum(prod, dim);"),
    "pairwise_drops_last": ("return orc_pairwise_sum(v, h) + orc_pairwise_sum(v + h, len - h);",
                            "return orc_pairwise_sum(v, h) + orc_pairwise_sum(v + h, len - h - 1);"),
    "observable_overwrites": ("for (int64_t i = 0; i < dim; ++i) lam[i] += terms[t].coeff * phi[i];",
                              "for (int64_t i = 0; i < dim; ++i) lam[i] = terms[t].coeff * phi[i];"),
    "gradient_factor_two_dropped": ("grad[g->param] += 2.0 * cfac * orc_pairwise_sum(im, dim);",
                                    "grad[g->param] += cfac * orc_pairwise_sum(im, dim);"),
    "gradient_sign": ("for (int64_t i = 0; i < dim; ++i) im[i] = cimag(conj(lam[i]) * phi[i]);",
                      "for (int64_t i = 0; i < dim; ++i) im[i] = cimag(lam[i] * conj(phi[i]));"),
    "gradient_ignores_controls": ("        if (!match) phi[i] = 0;\n", "        (void)match;\n"),
    "shift_generator_sign": ("case ORC_SHIFT: U[3] = 1; cfac = -1.0; break;", "case ORC_SHIFT: U[3] = 1; cfac = 1.0; break;"),
    "ry_generator_transposed": ("case ORC_RY: U[1] = -I; U[2] = I; cfac = 0.5; break;",
                                "case ORC_RY: U[1] = I; U[2] = -I; cfac = 0.5; break;"),
    "gradient_uncomputes_lambda_only": ("    orc_apply(psi, n, g->k, g->locs, U, g->nctrl, g->ctrl_locs, g->ctrl_vals);\n    orc_apply(lam,",
                                        "    orc_apply(lam,"),
    "splitmix_shift": ("z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;"),
    "splitmix_counter_off_by_one": ("u[i] = (double)(orc_splitmix64(seed, k0 + (uint64_t)i + 1) >> 11)",
                                    "u[i] = (double)(orc_splitmix64(seed, k0 + (uint64_t)i) >> 11)"),
    "sample_drops_imag": ("p[i] = r2 + i2;", "p[i] = r2;"),
    "sample_ties_go_left": ("if (nxt > t) { *acc = a; return j; }", "if (nxt >= t) { *acc = a; return j; }"),
    "collapse_not_normalised": ("psi[x] = r > 0 ? a / r : 1.0;", "psi[x] = r > 0 ? a : 1.0;"),
    "hadamard_sign_moved": ("U[0] = U[1] = U[2] = 1 / sqrt(2.0); U[3] = -1 / sqrt(2.0);",
                            "U[0] = U[2] = U[3] = 1 / sqrt(2.0); U[1] = -1 / sqrt(2.0);"),
    "y_sign": ("case ORC_Y: U[1] = -I; U[2] = I; break;", "case ORC_Y: U[1] = I; U[2] = -I; break;"),
    "phase_on_zero_only": ("case ORC_PHASE: U[0] = cexp(I * theta); U[3] = cexp(I * theta); break;",
                           "case ORC_PHASE: U[0] = cexp(I * theta); U[3] = 1; break;"),
    "pauli_z_sign": ("if (p == 3) { m[0][0] = 1; m[1][1] = -1; }", "if (p == 3) { m[0][0] = -1; m[1][1] = 1; }"),
    "rz_generator_sign": ("case ORC_RZ: U[0] = 1; U[3] = -1; cfac = 0.5; break;",
                          "case ORC_RZ: U[0] = -1; U[3] = 1; cfac = 0.5; break;"),
    "phase_generator_sign": ("case ORC_PHASE: U[0] = 1; U[3] = 1; cfac = -1.0; break;",
                             "case ORC_PHASE: U[0] = 1; U[3] = 1; cfac = 1.0; break;"),
    "rot_generator_factor": ("          cfac = 0.5;\n          break;", "          cfac = 1.0;\n          break;"),
    "gradient_controls_inverted": ("if ((((uint64_t)i >> g->ctrl_locs[c]) & 1u) != (uint64_t)g->ctrl_vals[c]) match = 0;",
                                   "if ((((uint64_t)i >> g->ctrl_locs[c]) & 1u) == (uint64_t)g->ctrl_vals[c]) match = 0;"),
    "dagger_in_forward_order": ("const orc_gate* g = &gates[dagger ? ngates - 1 - t : t];", "const orc_gate* g = &gates[t];"),
    "rot_paulis_reversed": ("for (int j = 0; j < k; ++j) {\n            cplx m[2][2];\n            pauli2(g->paulis[j], m);",
                            "for (int j = 0; j < k; ++j) {\n            cplx m[2][2];\n            pauli2(g->paulis[k - 1 - j], m);"),
    "sample_block_offset_dropped": ("int64_t b = b0 + walk(s0 + b0, b1 - b0, t, &acc);", "int64_t b = walk(s0 + b0, b1 - b0, t, &acc);"),
    "tdg_is_t": ("case ORC_TDG: U[0] = 1; U[3] = cexp(-I * M_PI / 4); break;", "case ORC_TDG: U[0] = 1; U[3] = cexp(I * M_PI / 4); break;"),
}


def _compile(name, text, out_dir):
    so = os.path.join(out_dir, f"lib_{name}.so")
    c = os.path.join(out_dir, f"{name}.c")
    with open(c, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fcx-limited-range", c, "-o", so, "-lm"], check=True, capture_output=True)
    return so


def _run_pins(so):
    env = dict(os.environ, QSIM_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    src = open(SRC).read()
    out_dir = str(tmp_path_factory.mktemp("mutants"))
    texts = {"unmodified": src}
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, f"mutant {name}: its text must occur exactly once in the oracle"
        texts[name] = src.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        libs = dict(zip(texts, ex.map(lambda kv: _compile(kv[0], kv[1], out_dir), texts.items())))
        return dict(zip(libs, ex.map(_run_pins, libs.values())))


def test_unmodified_oracle_passes_its_pins(outcomes):
    rc, tail = outcomes["unmodified"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(outcomes, name):
    rc, tail = outcomes[name]
    assert rc != 0, f"no pin fails with mutant {name}:\n{tail}"
