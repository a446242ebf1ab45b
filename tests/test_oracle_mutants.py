"""The oracle's pins must catch plausible mistakes: each mutant below plants one in a copy of the oracle's C source
(on the CPU, in a temporary directory), and the pin suite run against that copy must fail.

Each mutant is a mistake a reader of Section 3 could make: the sign of the warp, the direction of the beta test,
swapped gradient components, a backward difference, Eq. 3 without its factor 2, floor instead of nearest rounding
in Eq. 4, a neighbour window one short, the tie order of the sort, non-strict thresholds, h rounded down, clamping
instead of dropping samples outside the image, cos/sin swapped, Eq. 6 overwriting instead of accumulating, and, in
the backward warp of the registration step (Section 1), the wrong neighbour row or swapped horizontal / vertical
interpolation weights.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "warp_sign": ("out[n].w = g - v;", "out[n].w = g + v;"),
    "beta_direction": ("vb < srt[j].v", "srt[i].v < srt[j].v + p->beta"),
    "gradient_swap": ("float pcx = ex * c;", "float pcx = ey * c;"),
    "backward_difference": ("float ex = (x + 1 < W) ? dr(D, W, x + 1, y, r) - d : 0.0f;",
                            "float ex = (x >= 1) ? d - dr(D, W, x - 1, y, r) : 0.0f;"),
    "scan_length_no_factor_2": ("float twice = range * 2.0f;", "float twice = range;"),
    "floor_not_nearest": ("float rx = roundf(fx);", "float rx = floorf(fx);"),
    "window_one_short": ("int32_t half = p->N / 2;", "int32_t half = p->N / 2 - 1;"),
    "tie_order": ("return (a->k > b->k) - (a->k < b->k);", "return (a->k < b->k) - (a->k > b->k);"),
    "zeta_not_strict": ("fabsf(dw) < p->zeta", "fabsf(dw) <= p->zeta"),
    "gamma_not_strict": ("return e > gamma && dot > 0.0f;", "return e >= gamma && dot > 0.0f;"),
    "angle_not_strict": ("return e > gamma && dot > 0.0f;", "return e > gamma && dot >= 0.0f;"),
    "h_rounded_down": ("int32_t h = (L + 1) / 2;\n\n    memset", "int32_t h = L / 2;\n\n    memset"),
    "clamp_not_drop": ("if (!(rx >= 0.0f && rx < (float)W && ry >= 0.0f && ry < (float)H)) continue;",
                       "if (rx < 0) rx = 0; if (ry < 0) ry = 0; if (rx > W - 1) rx = W - 1; if (ry > H - 1) ry = H - 1;"),
    "cos_sin_swap": ("float ty = s * g;", "float ty = c * g;"),
    "mask_overwrites": ("O[srt[i].pix] += o;", "if (o) O[srt[i].pix] = o;"),
    "warp_wrong_neighbour_row": ("int64_t y1 = y0 + 1 < H ? y0 + 1 : y0;", "int64_t y1 = y0 > 0 ? y0 - 1 : y0;"),
    "warp_fx_fy_swap": ("out[i] = top + fy * (bot - top);", "out[i] = top + fx * (bot - top);"),
    "warp_weights_swap": ("float top = i00 + fx * (i01 - i00);\n            float bot = i10 + fx * (i11 - i10);",
                          "float top = i00 + fy * (i01 - i00);\n            float bot = i10 + fy * (i11 - i10);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "occ_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (tmp_path / "oracle" / "occ_oracle.c").write_text(src.replace(old, new, 1))
    (tmp_path / "tests").mkdir()
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    shutil.copy(os.path.join(ROOT, "scenes.py"), tmp_path / "scenes.py")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
