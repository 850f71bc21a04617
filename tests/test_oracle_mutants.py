"""The oracle's pins catch typical mistakes.

Each case plants one mistake (one or two edits) in a copy of
oracle/lv_oracle.c, builds it, and
runs tests/test_oracle_pins.py against that build in a child process: at
least one pin must fail.  The unchanged copy must pass them all.
"""
import os
import shutil
import subprocess
import sys

import pytest

from conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "lv_oracle.c")
OUT = os.path.join(ROOT, "tests", "_build", "mutants")

MUTANTS = {
    "none": None,
    # Eq. 4 without the -k_i a_C term of the target community
    "dropped gain term": ("const i128 G = ((i128)two_m * sc->e[c] - (i128)ki * a[c]) - s_old;",
                          "const i128 G = ((i128)two_m * sc->e[c]) - s_old;"),
    # Sec. 4.1 singlet rule blocking the wrong one of the two moves
    "flipped singlet rule": ("size[best] == 1 && best > ci) continue;",
                             "size[best] == 1 && best < ci) continue;"),
    # equal gains going to the larger label
    "flipped tie-break": ("(G == bestG && c < best)", "(G == bestG && c > best)"),
    # vertex following adding w(i,j) once instead of twice (R2)
    "VF weight": ("extra[j] += 2 * (int64_t)g->w[g->rowptr[i]];",
                  "extra[j] += (int64_t)g->w[g->rowptr[i]];"),
    # colouring in increasing instead of decreasing priority (R11)
    "colouring order": ("if (x->h != y->h) return x->h < y->h ? 1 : -1;",
                        "if (x->h != y->h) return x->h < y->h ? -1 : 1;"),
    # smallest degree first instead of largest (R11)
    "colouring degree order": ("if (x->d != y->d) return x->d < y->d ? 1 : -1;",
                               "if (x->d != y->d) return x->d < y->d ? -1 : 1;"),
    # the colouring degree counting the self-loop as a neighbour (R11)
    "colouring degree with loop": ("d += g->col[e] != v;", "d += 1;"),
    # a move on a zero gain
    "zero-gain move": ("if (bestG > 0) {", "if (bestG >= 0 && best != ci) {"),
    # the self-loop left out of e_in (R1)
    "self-loop out of e_in": ("if (C[g->col[e]] == C[i]) ein += g->w[e];",
                              "if (g->col[e] != i && C[g->col[e]] == C[i]) ein += g->w[e];"),
    # moves applied in place within a class (Gauss-Seidel instead of R6's Jacobi)
    "in-place moves": [("            sc->mv_v[nmoves] = i;\n            sc->mv_c[nmoves] = best;\n",
                        "            a[C[i]] -= k[i]; size[C[i]] -= 1; a[best] += k[i]; size[best] += 1;\n"
                        "            C[i] = best;\n"),
                       ("    for (int64_t t = 0; t < nmoves; ++t) {\n        const int32_t i = sc->mv_v[t]",
                        "    for (int64_t t = 0; t < 0; ++t) {\n        const int32_t i = sc->mv_v[t]")],
    # a coarse self-loop counting each intra edge once instead of per arc (R1)
    "coarse loop halved": ("            t[e].w = g->w[e];",
                           "            t[e].w = (t[e].u == t[e].v && u > g->col[e]) ? 0 : g->w[e];"),
    # coarse vertices numbered in descending instead of ascending label (R14)
    "descending renumbering": ("        for (int64_t c = 0; c < np; ++c) newid[c] = size[c] > 0 ? (int32_t)nn++ : -1;",
                               "        for (int64_t c = np - 1; c >= 0; --c) newid[c] = size[c] > 0 ? (int32_t)nn++ : -1;"),
    # the stop test on the absolute change (R9 reads it signed)
    "absolute stop test": ("    if (abs_mode) d = abs64(d);", "    d = abs64(d);"),
    # vertex following removing the larger end of an isolated edge (R3)
    "VF keeps the smaller end": ("if (deg1[j] && j < i) continue;", "if (deg1[j] && j > i) continue;"),
    # recursive VF testing the bound without the self-loop in k_i (R23)
    "recursive VF loop out of k": ("const int64_t k = wij + loop;", "const int64_t k = wij;"),
    # recursive VF keeping the smaller of a facing pair (R3 applied to R23)
    "recursive VF pair rule": ("!(target[j] == (int32_t)i && j < i)",
                               "!(target[j] == (int32_t)i && j > i)"),
    # coloured phases using the fine threshold and uncoloured ones the coarse (R12)
    "thresholds swapped": ("? prm->theta_high\n", "? prm->theta_low + 0.0 * prm->theta_high\n"),
    # the comparison of Sec. 5 counting pairs together only in p as FN and
    # only in s as FP (R22)
    "FP and FN swapped": [("else if (same_p) ++fp;", "else if (same_p) ++fn;"),
                          ("else if (same_s) ++fn;", "else if (same_s) ++fp;")],
    # symmetry accepting a mirror arc of another weight (Sec. 2)
    "mirror weight ignored": ("return lo < rowptr[j + 1] && col[lo] == i && w[lo] == wt;",
                              "return lo < rowptr[j + 1] && col[lo] == i;"),
    # a repeated column reported as an unsorted row
    "duplicate as ARG": ("if (col[e] == col[e - 1]) st = worse(st, ORC_ERR_DUPLICATE);",
                         "if (col[e] == col[e - 1]) st = worse(st, ORC_ERR_ARG);"),
    # a self-loop counted twice in k (R1 counts it once)
    "loop twice in k": ("for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) s += g->w[e];",
                        "for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e)\n"
                        "            s += g->col[e] == i ? 2 * (int64_t)g->w[e] : g->w[e];"),
}


def _build(name, change):
    src = open(SRC).read()
    for old, new in ([] if change is None else [change] if isinstance(change, tuple) else change):
        assert src.count(old) == 1, f"{name}: the line to change is gone"
        src = src.replace(old, new)
    os.makedirs(OUT, exist_ok=True)
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    c_path = os.path.join(OUT, f"{tag}.c")
    so_path = os.path.join(OUT, f"{tag}.so")
    with open(c_path, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", so_path, c_path])
    return so_path


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_planted_mistake(name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    so = _build(name, MUTANTS[name])
    env = dict(os.environ, LV_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    if name == "none":
        assert r.returncode == 0, r.stdout[-2000:]
    else:
        assert r.returncode == 1, (r.returncode, r.stdout[-2000:])  # a pin failed, nothing crashed
