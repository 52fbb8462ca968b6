"""The oracle's pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a wrong sign, a swapped index or
constant) in a copy of the oracle on the CPU, rebuilds the copy and runs the
pin suite against it; the suite must fail.  The real oracle is never touched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C = "oracle/dgs_oracle.c"
PY = "oracle/__init__.py"

# (name, file, text as it stands, planted mistake); the text occurs once.
MUTATIONS = [
    ("dilation dropped (Section 7.4 low-pass)", C,
     "f->a2 = S2[0] + 0.3; f->b2 = S2[1]; f->c2 = S2[3] + 0.3;",
     "f->a2 = S2[0]; f->b2 = S2[1]; f->c2 = S2[3];"),
    ("sign of the conic cross term", C,
     "        double pw = -0.5 * (r->A * dx * dx + r->Cc * dy * dy) - r->B * dx * dy;\n"
     "        double pmag",
     "        double pw = -0.5 * (r->A * dx * dx + r->Cc * dy * dy) + r->B * dx * dy;\n"
     "        double pmag"),
    ("transmittance dropped from compositing (Eq. 3 render)", C,
     "for (int ch = 0; ch < 3; ++ch) C[ch] += r->rgb[ch] * alpha * T;",
     "for (int ch = 0; ch < 3; ++ch) C[ch] += r->rgb[ch] * alpha;"),
    ("early-stop threshold", C,
     "        if (Tn < 1e-4) break;\n        for (int ch = 0; ch < 3; ++ch) C[ch]",
     "        if (Tn < 1e-3) break;\n        for (int ch = 0; ch < 3; ++ch) C[ch]"),
    ("cos and sin of the temporal basis swapped (Eq. 1)", C,
     "(k % 2 == 0) ? cos(", "(k % 2 == 1) ? cos("),
    ("closure ignores a missing layer (Section 4)", C,
     "if (!((mask[b >> 5] >> (b & 31)) & 1u)) break;",
     "if (!((mask[b >> 5] >> (b & 31)) & 1u)) { ++d; continue; }"),
    ("refinement layers off by one (Section 3)", C,
     "    for (int l = 1; l < d; ++l) {\n        for (int k = 0; k < 3; ++k) { a->mu[k]",
     "    for (int l = 1; l <= d && l < s->n_layers; ++l) {\n        for (int k = 0; k < 3; ++k) { a->mu[k]"),
    ("opacity clamp of the forward at 0.999 instead of 0.99", C,
     "        double alpha = araw < 0.99 ? araw : 0.99;\n        if (fabs(araw - 0.99)",
     "        double alpha = araw < 0.999 ? araw : 0.999;\n        if (fabs(araw - 0.99)"),
    ("alpha threshold of the forward at 1/128 instead of 1/255", C,
     "        if (alpha < 1.0 / 255.0) continue;\n        if (edge) mg = 1;",
     "        if (alpha < 1.0 / 128.0) continue;\n        if (edge) mg = 1;"),
    ("temporal basis frequency off by one (Eq. 1)", C,
     "int j = k / 2 + 1;", "int j = k / 2 + 2;"),
    ("Jacobian clamp factor", C,
     "double limx = 1.3 * (0.5 * cam->width) / cam->fx, limy = 1.3 * (0.5 * cam->height) / cam->fy;",
     "double limx = 1.1 * (0.5 * cam->width) / cam->fx, limy = 1.1 * (0.5 * cam->height) / cam->fy;"),
    ("conic-to-covariance adjoint sign", C,
     "for (int c = 0; c < 2; ++c) GS[2 * r + c] = -(QG[2 * r] * Q[c] + QG[2 * r + 1] * Q[2 + c]);",
     "for (int c = 0; c < 2; ++c) GS[2 * r + c] = (QG[2 * r] * Q[c] + QG[2 * r + 1] * Q[2 + c]);"),
    ("off-diagonal conic gradient not halved", C,
     "double G[4] = {g->A, 0.5 * g->B, 0.5 * g->B, g->Cc};", "double G[4] = {g->A, g->B, g->B, g->Cc};"),
    ("covariance factor gradient missing the factor 2", C,
     "            gM[3 * r + c] = 2.0 * acc;", "            gM[3 * r + c] = acc;"),
    ("mean2d adjoint: depth term sign", C,
     "gp[2] += -g->mx * fx * x / z2 - g->my * fy * y / z2;", "gp[2] += g->mx * fx * x / z2 - g->my * fy * y / z2;"),
    ("opacity adjoint misses the Gaussian factor", C,
     "g->o += galpha * ex[q];", "g->o += galpha;"),
    ("suffix term of the alpha adjoint not divided by (1 - alpha)", C,
     "galpha += gC[ch] * (r->rgb[ch] * T_q - suffix[ch] / (1.0 - alpha));",
     "galpha += gC[ch] * (r->rgb[ch] * T_q - suffix[ch]);"),
    ("sign of the cross term in the mean adjoint", C,
     "g->mx += gpw * (-(r->A * dx + r->B * dy));", "g->mx += gpw * (-(r->A * dx - r->B * dy));"),
    ("sigmoid derivative truncated", C,
     "double glogit = g->o * rec.o * (1.0 - rec.o);", "double glogit = g->o * rec.o;"),
    ("straight-through gradient ignores clipping", C,
     "if (!cl) gr[k] += gv[k];", "gr[k] += gv[k];"),
    ("affine interpolation weights swapped (Eq. 1)", C,
     "A[k] = (1.0 - *w) * a0[k] + *w * a1[k];", "A[k] = *w * a0[k] + (1.0 - *w) * a1[k];"),
    ("quantized decode uses the wrong step index", C,
     "return (double)s->res_q[o] * (double)s->res_step[(size_t)(l - 1) * K + k];",
     "return (double)s->res_q[o] * (double)s->res_step[(size_t)(l - 1) * K];"),
    ("derived bound of an early-stop flip dropped", C,
     "        if (fabs(Tn - 1e-4) <= (eps->rel_T + 1.01 * flip_a) * 1e-4) bnd += T * 2.0 * M;",
     "        if (fabs(Tn - 1e-4) <= (eps->rel_T + 1.01 * flip_a) * 1e-4) bnd += 0.0;"),
    ("derived bound of an alpha-threshold flip too small", C,
     "            const double a = (1.0 / 255.0) * (1.0 + eps->rel_alpha);",
     "            const double a = (1.0 / 255.0) * 0.1;"),
    ("derived bound of a depth-order swap too small", C,
     "            bnd += T_prev * a_prev * alpha * 2.0 * M;",
     "            bnd += T_prev * a_prev * alpha * 0.2 * M;"),
    ("SSIM constants swapped in the structure term", PY,
     "a1, a2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C2",
     "a1, a2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C1"),
    ("SSIM window sigma", PY,
     "def ssim_window(size: int = 11, sigma: float = 1.5)",
     "def ssim_window(size: int = 11, sigma: float = 1.0)"),
    ("sample instead of population standard deviation (Eq. 4)", PY,
     "std = float(np.sqrt(np.mean((x - mean) ** 2)))",
     "std = float(np.sqrt(np.sum((x - mean) ** 2) / max(x.size - 1, 1)))"),
    ("quantile position q M instead of q (M - 1) (Eq. 4)", PY,
     "h = q * (x.size - 1)", "h = min(q * x.size, x.size - 1)"),
    ("CVaR over the lower tail (Eq. 2)", PY,
     "top = np.argsort(-D, kind=\"stable\")[:k]", "top = np.argsort(D, kind=\"stable\")[:k]"),
    ("prefix hinge with the wrong orientation (Eq. 2)", PY,
     "            if D[j] > D[i]:\n                M += (D[j] - D[i]) / len(pairs_m)",
     "            if D[i] > D[j]:\n                M += (D[i] - D[j]) / len(pairs_m)"),
    ("mean and quantile weights swapped in the risk-adjusted utility (Eq. 4)", PY,
     "((1.0 - alpha) * mean + alpha * quant) / (1.0 + beta * std)",
     "(alpha * mean + (1.0 - alpha) * quant) / (1.0 + beta * std)"),
    ("CVaR weight spread over all states instead of the tail (Eq. 2)", PY,
     "w[top] += lambda_c / k", "w[top] += lambda_c / S"),
    ("anchor gradient weight (Eq. 2)", PY,
     "w[s] += anchor_weight / len(anchors)", "w[s] += anchor_weight"),
    ("SSIM gradient: covariance term halved", PY,
     "d_exy = 2 * f / a2", "d_exy = f / a2"),
    ("SSIM gradient: variance term sign", PY,
     "d_exx = -f / b2", "d_exx = f / b2"),
    ("temporal-change gradient sign (Eq. 2)", PY,
     "            grad[j] += gf\n            grad[i] -= gf",
     "            grad[j] -= gf\n            grad[i] += gf"),
]


def _copy_tree(dst):
    ign = shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__", "csrc", "_build*")
    for d in ("oracle", "tests", "paper_2606_17212_b300"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d), ignore=ign)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)


def test_mutation_sites_exist():
    for name, path, old, _ in MUTATIONS:
        with open(os.path.join(ROOT, path)) as f:
            assert f.read().count(old) == 1, name


@pytest.mark.parametrize("name,path,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, path, old, new):
    _copy_tree(str(tmp_path))
    p = os.path.join(str(tmp_path), path)
    with open(p) as f:
        text = f.read()
    assert text.count(old) == 1, name
    with open(p, "w") as f:
        f.write(text.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "8"))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                        "-p", "no:randomly"], cwd=str(tmp_path), env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)
    tail = r.stdout.strip().splitlines()[-3:]
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.returncode, tail)
