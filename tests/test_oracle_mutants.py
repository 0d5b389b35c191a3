"""The pins catch plausible mistakes in the oracle.  Each mutant plants one error in a copy of
oracle/gs_oracle.c -- a dropped term, a wrong sign, a transposed operand, a wrong clamp, an
off-by-one, a decision that is not listed or not flipped -- compiles it on the CPU, and runs
the pins that should notice it against that library (GS_ORACLE_LIB); every mutant must make
them fail.  Nothing here touches the CUDA path."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gs_oracle.c")
PINS = "tests/test_oracle_pins.py"
DEC = "tests/test_oracle_decisions.py"

# (name, original text, mutated text, pins that must fail)
MUTANTS = [
    # arithmetic of the definition (Sec. 4, App. A, App. C, SH basis)
    ("rotation: transposed off-diagonal", "R[1] = 2.0 * (i * j - r * k);", "R[1] = 2.0 * (i * j + r * k);",
     [f"{PINS}::test_quat_rotation_matches_rodrigues"]),
    ("SH: Condon-Shortley phase dropped", "double sign = (m % 2) ? -1.0 : 1.0;", "double sign = 1.0;",
     [f"{PINS}::test_sh_basis_matches_scipy", f"{PINS}::test_sh_basis_matches_published_constants"]),
    ("EWA: low-pass dilation dropped", "g->cov2[0] = S00 + cfg->dilation;", "g->cov2[0] = S00;",
     [f"{PINS}::test_ewa_isotropic_on_axis_closed_form"]),
    ("blend: 0.99 clamp dropped", "const double alpha = clamped ? cfg->alpha_max : oG;", "const double alpha = oG;",
     [f"{PINS}::test_opacity_clamp_gives_99_percent"]),
    ("backward: sign of dL/du", "p->uv[0] = (g->conic[0] * c->dx + g->conic[1] * c->dy) * dL_dpower;",
     "p->uv[0] = -(g->conic[0] * c->dx + g->conic[1] * c->dy) * dL_dpower;",
     [f"{PINS}::test_backward_matches_finite_differences_tiny"]),
    # the decision machinery (which decisions are listed, how each is flipped, the allowance)
    ("stop decision not listed", "            ADD_DEC(DEC_STOP, gi, -1);", "            ;",
     [f"{DEC}::test_stop_near_threshold_is_flagged_and_the_allowance_is_the_real_gradient_change"]),
    ("only equal depth keys listed", "key - prev_key <= 1u", "key == prev_key",
     [f"{DEC}::test_adjacent_depth_keys_are_flagged_and_the_alternative_swaps_them"]),
    ("skip flip not applied", "if (flips(flip, DEC_SKIP, gi)) skip = !skip;", ";",
     [f"{DEC}::test_skip_near_threshold_is_flagged_and_its_alternative_is_the_other_side"]),
    ("clamp flip not applied", "if (flips(flip, DEC_CLAMP, gi)) clamped = !clamped;", ";",
     [f"{DEC}::test_clamp_near_threshold_is_flagged_with_its_derivative_switched"]),
    ("Gaussians outside the list not listed",
     "power_margin(g, dx, dy, cfg))) ADD_DEC(DEC_ADD, gi, -1);", "power_margin(g, dx, dy, cfg))) {}",
     [f"{DEC}::test_tile_membership_near_the_radius_rounding_is_flagged"]),
    ("radius alternative off by one", "r_alt[1] = g->radius + 1;", "r_alt[1] = (int)floor(rr) + 1;",
     [f"{DEC}::test_tile_membership_near_the_radius_rounding_is_flagged"]),
    ("power margin on |P| instead of the terms' magnitude sum",
     "double Q = 0.5 * (fabs(g->conic[0]) * dx * dx + fabs(g->conic[2]) * dy * dy) + fabs(g->conic[1] * dx * dy);",
     "double Q = fabs(0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) + g->conic[1] * dx * dy);",
     [f"{DEC}::test_power_margin_follows_the_conditioning_of_the_quadratic_form"]),
    ("allowance: sum instead of difference", "d.op = (take2 ? p2[b].op : 0.0) - (take1 ? p1[a].op : 0.0);",
     "d.op = (take2 ? p2[b].op : 0.0) + (take1 ? p1[a].op : 0.0);",
     [f"{DEC}::test_stop_near_threshold_is_flagged_and_the_allowance_is_the_real_gradient_change",
      f"{DEC}::test_clamp_near_threshold_is_flagged_with_its_derivative_switched"]),
    ("colour-clamp allowance dropped", "if (!(g->rgb_amb & (1u << ch)) || d_rgb[3 * i + ch] == 0.0) continue;",
     "continue;", [f"{DEC}::test_colour_clamp_near_zero_adds_that_channels_terms_to_the_allowance"]),
]


def _run(mutant, workdir):
    name, old, new, pins = mutant
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the mutated text must occur exactly once"
    base = os.path.join(workdir, "m%d" % MUTANTS.index(mutant))
    with open(base + ".c", "w") as f:
        f.write(src.replace(old, new))
    cc = subprocess.run(["gcc", "-O1", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                         base + ".c", "-o", base + ".so", "-lm"], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    env = dict(os.environ, GS_ORACLE_LIB=base + ".so", OMP_NUM_THREADS="2")
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *pins],
                         cwd=ROOT, env=env, capture_output=True, text=True)
    return name, res.returncode, res.stdout[-600:]


def test_every_mutant_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp, cf.ThreadPoolExecutor(max_workers=4) as pool:
        results = list(pool.map(lambda m: _run(m, tmp), MUTANTS))
    survivors = [(name, out) for name, rc, out in results if rc != 1]
    assert not survivors, survivors


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutated_text_is_present(mutant):
    assert open(SRC).read().count(mutant[1]) == 1
