"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a temporary copy of the oracle source (CPU only), rebuilds it and
checks that tests/test_oracle_pins.py fails on it; the real oracle is never
touched.  A mutation that survives would mean a part of the oracle is
unpinned."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    # level-3 approximate inverse 2b - b P b (Sec. II-A, recurrence for P_i)
    "drop_newton_level3": ("const double xd = 2.0 * beta[e] - beta[e] * Pd[ps + e] * beta[e];",
                           "const double xd = beta[e];"),
    # level-2 approximate inverse 2b - b T b (recurrence for T_i)
    "drop_newton_level2": ("const double xd = 2.0 * beta[a] - beta[a] * Td[ls + a] * beta[a];",
                           "const double xd = beta[a];"),
    # twist block m = floor((n-1)/2) (Algorithm 2)
    "twist_index_off_by_one": ("const int mz = (nz - 1) / 2;", "const int mz = nz / 2;"),
    # coupling of the lower half to the block below (Algorithm 4, reading R6)
    "alg4_wrong_coupling": ("rhs[e] -= L[i + e] * y[i + bs + e];", "rhs[e] -= L[i - bs + e] * y[i + bs + e];"),
    # the twist block takes both couplings (Algorithm 2)
    "twist_block_one_side": ("if (mid < nb - 1)\n            for (long e = 0; e < bs; ++e) rhs[e] -= L[cur + e] * y[cur + bs + e];", ""),
    # scalar pivot recurrence (recurrence for M_i)
    "pivot_sign": ("if (a > 0) v -= To[s + a - 1] * To[s + a - 1] / M[s + a - 1];",
                   "if (a > 0) v += To[s + a - 1] * To[s + a - 1] / M[s + a - 1];"),
    # x-band of C X C uses the x-neighbour's coupling
    "xband_wrong_neighbour": ("xk[e] -= C[e] * xo * C[e + 1];", "xk[e] -= C[e] * xo * C[e];"),
    # Algorithm 6 couples to the final x (reading R7)
    "alg6_uses_y": ("bp[e] = U[i + e] * x[i + bs + e];", "bp[e] = U[i + e] * y[i + bs + e];"),
    # level-3 filter vector in beta (definition of beta_i)
    "beta_level3_ignores_t": ("w[e] = C[e] * (t ? t[e] : 1.0);", "w[e] = C[e];"),
    # harmonic-mean face coefficient
    "arithmetic_mean_faces": ("return 2.0 * ka * kb / (ka + kb);", "return 0.5 * (ka + kb);"),
    # Dirichlet face half a cell from the centre
    "dirichlet_full_cell": ("else if (bc[0] == 0) diag += 2.0 * ka * ax;", "else if (bc[0] == 0) diag += ka * ax;"),
    # CG beta
    "cg_beta_inverted": ("else beta = rho_new / rho;", "else beta = rho / rho_new;"),
    # ILU(0) pivots keep only the lower-neighbour terms of the same block
    "ilu_ignores_block_split": ("if (iz > 0 && a - nxy >= lo) v -= cz[a - nxy] * cz[a - nxy] / D[a - nxy];",
                                "if (iz > 0) v -= cz[a - nxy] * cz[a - nxy] / D[a - nxy];"),
    # ILU(0) backward sweep divides by the pivot
    "ilu_backward_no_pivot": ("        z[a] -= v / D[a];", "        z[a] -= v;"),
    # combination: B_NTD acts on the residual of the smoother (Eq. (com))
    "combo_drops_residual": ("for (long e = 0; e < n; ++e) w[e] = r[e] - w[e];",
                             "for (long e = 0; e < n; ++e) w[e] = r[e];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "ffp_oracle.c")).read()
    assert old in src, f"mutation anchor for {name} not found in the oracle"
    work = tmp_path / "repo"
    for sub in ("oracle", "tests", "paper_1909_09771_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), work / sub,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    (work / "oracle" / "ffp_oracle.c").write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=work, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"


# Mistakes planted in the learned-filter oracle (oracle/convnet.py), caught by
# tests/test_oracle_convnet.py.
CONVNET_MUTATIONS = {
    # target weights theta_0 / theta_k, inverted
    "target_weights_inverted": ("acc += (theta[0] / theta[k]) * y * y",
                                "acc += (theta[k] / theta[0]) * y * y"),
    # each Ritz vector scaled to max |y| = 1 before it is weighted
    "target_no_normalisation": ("y = Y[:, k] / np.max(np.abs(Y[:, k]))", "y = Y[:, k]"),
    # the floor applies after scaling to max 1
    "target_floor_before_scaling": ("t = np.maximum(t / t.max(), floor)",
                                    "t = np.maximum(t, floor) / np.maximum(t, floor).max()"),
}


@pytest.mark.parametrize("name", sorted(CONVNET_MUTATIONS))
def test_convnet_pins_catch_planted_mistake(name, tmp_path):
    old, new = CONVNET_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "convnet.py")).read()
    assert old in src, f"mutation anchor for {name} not found in the convnet oracle"
    work = tmp_path / "repo"
    for sub in ("oracle", "tests", "paper_1909_09771_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), work / sub,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    (work / "oracle" / "convnet.py").write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_convnet.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=work, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"


# Mistakes planted in the oracle's X = beta form (FFP_SCHUR_BETA), caught by the
# dense construction of tests/test_reading_study.py.
SCHUR_BETA_MUTATIONS = {
    "beta_form_level3_uses_newton": ("dk[e] -= C[e] * (c->classic ? beta[e] : xd) * C[e];",
                                     "dk[e] -= C[e] * xd * C[e];"),
    "beta_form_level3_keeps_offdiagonals": ("        if (c->classic) continue;                         /* X = beta: diagonal only */\n", ""),
    "beta_form_level2_keeps_offdiagonal": ("if (a + 1 < nx && !c->classic) {", "if (a + 1 < nx) {"),
}


@pytest.mark.parametrize("name", sorted(SCHUR_BETA_MUTATIONS))
def test_dense_construction_catches_planted_mistake(name, tmp_path):
    old, new = SCHUR_BETA_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "ffp_oracle.c")).read()
    assert old in src, f"mutation anchor for {name} not found in the oracle"
    work = tmp_path / "repo"
    for sub in ("oracle", "tests", "paper_1909_09771_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), work / sub,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    (work / "oracle" / "ffp_oracle.c").write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_reading_study.py", "-q", "-x",
                        "-p", "no:cacheprovider", "-k", "dense_construction"], cwd=work,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived:\n{r.stdout[-2000:]}"
