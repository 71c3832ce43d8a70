"""Planted mistakes: each mutant of the oracle's C source (a flipped sign, a
dropped term, a wrong index or a transposed operand) must fail at least one
of the fast pins.  Mutants are compiled to a temporary library and run in a
subprocess, so a mutant that crashes also counts as caught."""
import os
import subprocess
import sys
import textwrap
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fv_oracle.c")

# (name, original text, mutated text); the original must occur exactly once
MUTANTS = [
    ("hll_diffusion_sign", "- apm * (R.u[q] - L.u[q])", "+ apm * (R.u[q] - L.u[q])"),
    ("hll_left_weight", "((ap * L.f[q] + am * R.f[q])", "((am * L.f[q] + am * R.f[q])"),
    ("wave_speed_sign", "max0(L.c - L.vn, R.c - R.vn)", "max0(L.c + L.vn, R.c - R.vn)"),
    ("sound_speed_gamma", "s->c = sqrt(gamma * w[4] / w[0]);", "s->c = sqrt(w[4] / w[0]);"),
    ("flux_pressure_dropped", "s->f[1 + axis] = s->f[1 + axis] + w[4];", "s->f[1 + axis] = s->f[1 + axis];"),
    ("energy_flux_pressure", "s->f[4] = (s->u[4] + w[4]) * vn;", "s->f[4] = s->u[4] * vn;"),
    ("minmod_min_to_max", "if (b < r) r = b;", "if (b > r) r = b;"),
    ("limiter_centred_diff", "0.5 * (d_minus + d_plus)", "0.5 * (d_minus - d_plus)"),
    ("pressure_ke_sign", "w[4] = (gamma - 1.0) * (u[4] - ke);", "w[4] = (gamma - 1.0) * (u[4] + ke);"),
    ("prim_to_cons_index", "+ mz * w[3]);", "+ mz * w[2]);"),
    ("recon_right_sign", "a->W[q][o] - 0.5 * a->S[q][o]", "a->W[q][o] + 0.5 * a->S[q][o]"),
    ("recon_left_cell", "a->W[q][ol] + 0.5 * a->S[q][ol]", "a->W[q][o] + 0.5 * a->S[q][ol]"),
    ("difference_shift", "a->W[q][o] - a->W[q][at_shift(m, i, j, k, axis, -1)]",
     "a->W[q][at_shift(m, i, j, k, axis, -1)] - a->W[q][o]"),
    ("update_y_sign", "acc = acc - (a->F[1][q]", "acc = acc + (a->F[1][q]"),
    ("update_z_spacing", "a->F[2][q][o]) * inv[2]", "a->F[2][q][o]) * inv[0]"),
    ("rk2_stage2_sign", "U[o] = 0.5 * ((old[o] + U[o]) + dU[o]);", "U[o] = 0.5 * ((old[o] + U[o]) - dU[o]);"),
    ("rk2_stage1_base", "U[o] = old[o] + dU[o];", "U[o] = U[o] + dU[o] + dU[o];"),
    ("dt_transposed_spacing", "(fabs(w[2]) + c) * idy", "(fabs(w[2]) + c) * idx"),
    ("ghost_outflow_index", "return g < 0 ? 0 : n - 1;", "return g < 0 ? 1 : n - 1;"),
    ("ghost_periodic_wrap", "return r < 0 ? r + n : r;", "return r < 0 ? r + n - 1 : r;"),
    ("fallback_wrong_cell", "wl[q] = a->W[q][ol];", "wl[q] = a->W[q][o];"),
    ("sum_volume", "out[q] = orc_pairwise_sum(v, n) * vol;", "out[q] = orc_pairwise_sum(v, n);"),
]

PINS = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}, {tests!r}]
    import oracle as orc
    import test_oracle_pointwise as tp, test_oracle_scheme as ts, test_oracle_physics as tph
    checks = [
        lambda: tp.test_cons_prim_closed_form(orc),
        lambda: tp.test_limiter_extremum_and_first_order(orc),
        lambda: tp.test_hll_consistency(orc),
        lambda: tp.test_hll_matches_textbook_form(orc),
        lambda: ts.test_ghost_fill_matches_numpy_pad(orc, (0, 0, 0)),
        lambda: ts.test_ghost_fill_matches_numpy_pad(orc, (1, 1, 1)),
        lambda: ts.test_dt_uniform_closed_form(orc),
        lambda: ts.test_conservation_periodic_roundoff(orc),
        lambda: ts.test_conserved_sums_volume(orc),
        lambda: ts.test_axis_permutation(orc, 2),
        lambda: ts.test_face_fallback_near_vacuum(orc),
        lambda: tph.test_sod_star_plateau(orc),
        lambda: tph.test_smooth_wave_orders(orc),
    ]
    failed = 0
    for c in checks:
        try:
            c()
        except Exception:
            failed += 1
    print("failed", failed)
    sys.exit(1 if failed else 0)
""")


def _run_pins(lib_path, tmp_path):
    script = tmp_path / "pins.py"
    script.write_text(PINS.format(root=ROOT, tests=os.path.join(ROOT, "tests")))
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=str(lib_path))
    return subprocess.run([sys.executable, str(script)], env=env, capture_output=True,
                          text=True, timeout=600)


def _compile(src_text, tmp_path, name):
    c = tmp_path / f"{name}.c"
    c.write_text(src_text)
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared",
                    "-I", os.path.join(ROOT, "oracle"), "-o", str(so), str(c), "-lm"],
                   check=True)
    return so


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """Compile the control and every mutant, run the pins on all of them in
    parallel subprocesses; returns name -> CompletedProcess."""
    src = open(SRC).read()
    jobs = {"control": src}
    for name, orig, mut in MUTANTS:
        assert src.count(orig) == 1, f"mutation site for {name} not unique"
        jobs[name] = src.replace(orig, mut)

    def run(item):
        name, text = item
        d = tmp_path_factory.mktemp(name)
        return name, _run_pins(_compile(text, d, name), d)

    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        return dict(ex.map(run, jobs.items()))


def test_unmutated_oracle_passes_the_pin_harness(mutant_results):
    r = mutant_results["control"]
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(mutant_results, name):
    r = mutant_results[name]
    assert r.returncode != 0, f"mutant {name} survived: {r.stdout}"
