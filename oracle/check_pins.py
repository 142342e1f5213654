"""Mutation check of the oracle's pins (maintainer tool; not collected by pytest).

The oracle is pinned by tests that do not call it for their expected values
(closed forms, inverse maps, brute force, central differences, hand-computed
codes).  To show that those pins would notice a plausible mistake, this plants
one mistake at a time in the oracle's sources -- a dropped term, a wrong sign,
index or exponent, a transposed factor, a removed clamp, truncation or skip --
runs the pin tests (the oracle-written golden file left out) and reports
whether they fail.  Every source is restored after each run (and at start-up,
if an earlier run was interrupted).

    python -m oracle.check_pins            # all mutations
    python -m oracle.check_pins "no SH"    # those whose label contains the text

A mutation that makes the march stop advancing shows up as a timeout (the
suite's per-test timeout turns it into a failure in a normal run).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BACKUP = os.path.join(ROOT, "oracle", "_build", "check_pins_backup")
PINS = ["tests/test_oracle_render.py", "tests/test_oracle_grad.py", "tests/test_oracle_geometry.py",
        "tests/test_oracle_sh.py", "tests/test_oracle_losses.py", "tests/test_oracle_morton.py",
        "tests/test_oracle_sg.py", "tests/test_oracle_image_loss.py"]

# (file, label, original text, planted text)
MUTATIONS = [
    ('oracle/rgx_oracle.c', 'no half-pixel in u',
     '((double)u + 0.5 - cam->cx)',
     '((double)u + 0.0 - cam->cx)'),
    ('oracle/rgx_oracle.c', 'fx/fy swapped',
     '- cam->cx) / cam->fx, ((double)v + 0.5 - cam->cy) / cam->fy',
     '- cam->cx) / cam->fy, ((double)v + 0.5 - cam->cy) / cam->fx'),
    ('oracle/rgx_oracle.c', 'exit too early',
     '    if (t1 < t0 || t1 < tn) return tn;\n    return t1;',
     '    if (t1 < t0 || t1 < tn) return tn;\n    return tn + 0.8 * (t1 - tn);'),
    ('oracle/rgx_oracle.c', 'box without truncation radius',
     'double st = sqrt(P[l].Qe) * P[l].s[j];',
     'double st = P[l].s[j];'),
    ('oracle/rgx_oracle.c', 'end-point samples',
     'double t = tS + (k + 0.5) * dtk;',
     'double t = tS + (k + 1.0) * dtk;'),
    ('oracle/rgx_oracle.c', 'no hard truncation',
     'if (!(q <= p->Qe)) continue;      /* hard truncation */',
     '/* none */'),
    ('oracle/rgx_oracle.c', 'density exp(-q)',
     'double g = p->sig * exp(-0.5 * q);',
     'double g = p->sig * exp(-q);'),
    ('oracle/rgx_oracle.c', 'C without T',
     'out->C[r] += out->T * alpha * ci[r];',
     'out->C[r] += alpha * ci[r];'),
    ('oracle/rgx_oracle.c', 'Eq5 T^(+1/3)',
     'a *= pow(out->T, -1.0 / 3.0);',
     'a *= pow(out->T, 1.0 / 3.0);'),
    ('oracle/rgx_oracle.c', 'Eq5 no T factor',
     'a *= pow(out->T, -1.0 / 3.0);',
     'a *= 1.0;'),
    ('oracle/rgx_oracle.c', 'Eq5 t*beta',
     'double a = tS / op->beta;',
     'double a = tS * op->beta / 1e6;'),
    ('oracle/rgx_oracle.c', 'closest hit needs tin>ta',
     'if (ch[i].tout > ta && ch[i].tin < tf) {',
     'if (ch[i].tin > ta && ch[i].tin < tf) {'),
    ('oracle/rgx_oracle.c', 'hit set drops enclosing chords',
     'if (ch[i].tin < tcut && ch[i].tout > tS) hits[nh++] = i;',
     'if (ch[i].tin < tcut && ch[i].tin >= tS) hits[nh++] = i;'),
    ('oracle/rgx_oracle.c', 'no SH offset',
     'double acc = 0.5;',
     'double acc = 0.0;'),
    ('oracle/rgx_oracle.c', 'no colour clamp',
     'c[r] = pre[r] > 0 ? pre[r] : 0;',
     'c[r] = pre[r];'),
    ('oracle/losses.py', 'SSIM constants swapped',
     'SSIM_WIN, SSIM_SIGMA, SSIM_C1, SSIM_C2 = 11, 1.5, 0.01 ** 2, 0.03 ** 2',
     'SSIM_WIN, SSIM_SIGMA, SSIM_C1, SSIM_C2 = 11, 1.5, 0.03 ** 2, 0.01 ** 2'),
    ('oracle/losses.py', 'SSIM window sigma 1',
     'SSIM_WIN, SSIM_SIGMA, SSIM_C1, SSIM_C2 = 11, 1.5, 0.01 ** 2, 0.03 ** 2',
     'SSIM_WIN, SSIM_SIGMA, SSIM_C1, SSIM_C2 = 11, 1.0, 0.01 ** 2, 0.03 ** 2'),
    ('oracle/losses.py', 'SSIM grad drops the 2 x_p factor',
     'dS = (_blur(a, w1) + 2.0 * x * _blur(b, w1) + y * _blur(c, w1)) / n',
     'dS = (_blur(a, w1) + x * _blur(b, w1) + y * _blur(c, w1)) / n'),
    ('oracle/losses.py', 'SSIM covariance sign',
     'vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my',
     'vx, vy, cxy = exx - mx * mx, eyy - my * my, exy + mx * my'),
    ('oracle/losses.py', 'L1 gradient sign',
     'g = (1.0 - lam) * np.sign(x - y) / n - lam * dS',
     'g = (1.0 - lam) * np.sign(y - x) / n - lam * dS'),
    ('oracle/rgx_oracle.c', 'SG lobe without -1',
     'return exp(r[3] * (cd - 1.0));',
     'return exp(r[3] * cd);'),
    ('oracle/rgx_oracle.c', 'SG sharpness sign',
     'return exp(r[3] * (cd - 1.0));',
     'return exp(-r[3] * (cd - 1.0));'),
    ('oracle/rgx_oracle.c', 'SG axis not normalised',
     'double cd = (r[0]*d[0] + r[1]*d[1] + r[2]*d[2]) / nu;',
     'double cd = (r[0]*d[0] + r[1]*d[1] + r[2]*d[2]);'),
    ('oracle/rgx_oracle.c', 'SG amplitude channels reversed',
     'pre[r] += p->sg[7*j + 4 + r] * e;',
     'pre[r] += p->sg[7*j + 6 - r] * e;'),
    ('oracle/rgx_oracle.c', 'SG axis gradient not projected',
     'atomic_add(&gj[c], (dmu[c] - mu[c]*md) / nu);',
     'atomic_add(&gj[c], dmu[c] / nu);'),
    ('oracle/rgx_oracle.c', 'SG sharpness gradient without -1',
     'atomic_add(&gj[3], sa * e * (cosv - 1.0));',
     'atomic_add(&gj[3], sa * e * cosv);'),
    ('oracle/rgx_oracle.c', 'SG gradient ignores the clamp',
     'm[c] = pre[c] > 0 ? dcl[q][c] : 0.0;',
     'm[c] = dcl[q][c];'),
    ('oracle/rgx_oracle.c', 'no lattice guard (first)',
     'int64_t jj = (int64_t)floor((th - tn) / op->dt) - 1;\n                j = jj > 0 ? jj : 0;',
     'int64_t jj = (int64_t)floor((th - tn) / op->dt);\n                j = jj > 0 ? jj : 0;'),
    ('oracle/rgx_oracle.c', 'termination ignores T',
     'while (tS < tf && out->T > op->t_eps) {',
     'while (tS < tf) {'),
    ('oracle/rgx_oracle.c', 'skip ignores empty segment',
     'if (nh == 0) {\n                if (op->skip) {',
     'if (nh == 0) {\n                if (0) {'),
    ('oracle/rgx_oracle.c', 'no bg/opacity term',
     'dsig = s->dtk * (dsig - dTf * r.T);',
     'dsig = s->dtk * dsig;'),
    ('oracle/rgx_oracle.c', 'T instead of T_next',
     'dsig += a[c] * (Tn * s->c[c] - (r.C[c] - Cle[c]));',
     'dsig += a[c] * (s->T * s->c[c] - (r.C[c] - Cle[c]));'),
    ('oracle/rgx_oracle.c', 'colour weight without T',
     'double dci[3] = { a[0]*w, a[1]*w, a[2]*w };',
     'double dci[3] = { a[0]*alpha, a[1]*alpha, a[2]*alpha };'),
    ('oracle/rgx_oracle.c', 'density grad without 1/sig',
     'atomic_add(&g_dens[cb->l], wg / pr->sig);',
     'atomic_add(&g_dens[cb->l], wg);'),
    ('oracle/rgx_oracle.c', 'mean grad sign',
     'atomic_add(&g_means[3*cb->l + k], wg * v);',
     'atomic_add(&g_means[3*cb->l + k], -wg * v);'),
    ('oracle/rgx_oracle.c', 'dM transposed',
     'atomic_add(&gM[9*cb->l + 3*j + k], -wg * y[j] * xm[k]);',
     'atomic_add(&gM[9*cb->l + 3*j + k], -wg * y[k] * xm[j]);'),
    ('oracle/rgx_oracle.c', 'scale chain transposed',
     'ds += G[3*j + k] * (-pr->R[3*k + j] / (pr->s[j] * pr->s[j]));',
     'ds += G[3*j + k] * (-pr->R[3*j + k] / (pr->s[j] * pr->s[j]));'),
    ('oracle/rgx_oracle.c', 'SH grad ignores clamp',
     'if (pre[c] > 0) atomic_add(',
     'if (1) atomic_add('),
    ('oracle/rgx_oracle.c', 'quat grad no projection',
     'g_quats[4*l + 0] += (dw - w*dot) / nq;',
     'g_quats[4*l + 0] += dw / nq;'),
    ('oracle/rgx_oracle.c', 'colour grad without g/sigma',
     'for (int c = 0; c < 3; c++) dcl[slot][c] += dci[c] * cb->g / s->sigma;',
     'for (int c = 0; c < 3; c++) dcl[slot][c] += dci[c];'),
    ('oracle/rgx_oracle.c', 'M transposed',
     'p->M[3*j + k] = p->R[3*k + j] / s[j];',
     'p->M[3*j + k] = p->R[3*j + k] / s[j];'),
    ('oracle/rgx_oracle.c', 'M times s',
     'p->M[3*j + k] = p->R[3*k + j] / s[j];',
     'p->M[3*j + k] = p->R[3*k + j] * s[j];'),
    ('oracle/rgx_oracle.c', 'Q_eps without 2',
     'p->Qe = (sig > sigma_eps) ? 2.0 * log(sig / sigma_eps) : 0.0;',
     'p->Qe = (sig > sigma_eps) ? log(sig / sigma_eps) : 0.0;'),
    ('oracle/rgx_oracle.c', 'no Condon-Shortley phase',
     'pmm *= -f * sx;',
     'pmm *= f * sx;'),
    ('oracle/rgx_oracle.c', 'SH norm 2pi',
     'double K = sqrt((2.0*l + 1.0) / (4.0 * M_PI)',
     'double K = sqrt((2.0*l + 1.0) / (2.0 * M_PI)'),
    ('oracle/rgx_oracle.c', 'cos/sin swapped',
     'if (m > 0) v = sqrt(2.0) * K * cos(am * phi) * P;\n            else if (m < 0) v = sqrt(2.0) * K * sin(am * phi) * P;',
     'if (m > 0) v = sqrt(2.0) * K * sin(am * phi) * P;\n            else if (m < 0) v = sqrt(2.0) * K * cos(am * phi) * P;'),
    ('oracle/rgx_oracle.c', 'chord exit too far',
     '*tout = (-b + sq) / a;',
     '*tout = (-b + 1.01 * sq) / a;'),
    ('oracle/rgx_oracle.c', 'rotation sign',
     'R[1] = 2*(x*y - w*z);',
     'R[1] = 2*(x*y + w*z);'),
    ('oracle/rgx_oracle.c', 'Legendre recurrence',
     'pll = ((2*ll - 1) * x * pm1 - (ll + m - 1) * pmm) / (ll - m);',
     'pll = ((2*ll - 1) * x * pm1 - (ll + m) * pmm) / (ll - m);'),
    ('oracle/rgx_oracle.c', 'box without rotation',
     'acc += P[l].R[3*i+j] * P[l].R[3*i+j] * st * st;',
     'acc += (i == j) * st * st;'),
    ('oracle/losses.py', 'bound constant',
     'K_BOUND = 2.0 / (math.pi * math.sqrt(3.0))',
     'K_BOUND = 2.0 / (math.pi * math.sqrt(2.0))'),
    ('oracle/losses.py', 'loss gradient',
     'dr = r[:, None] * (3.0 * s / ss - 1.0 / s)',
     'dr = r[:, None] * (2.0 * s / ss - 1.0 / s)'),
    ('oracle/losses.py', 'loss not averaged',
     'loss = float(np.where(over, r - r0, 0.0).sum() / n)',
     'loss = float(np.where(over, r - r0, 0.0).sum())'),
    ('oracle/losses.py', 'densify times f',
     '/ float(focal)',
     '* float(focal)'),
    ('oracle/losses.py', 'densify counts unseen',
     'seen = gn > 0',
     'seen = gn >= 0'),
    ('oracle/morton.py', 'interleave z most significant',
     'for axis, off in ((0, 2), (1, 1), (2, 0)):',
     'for axis, off in ((0, 0), (1, 1), (2, 2)):'),
    ('oracle/morton.py', 'quantise no clip',
     'cell = np.clip(cell, 0, (1 << bits) - 1)',
     'cell = np.clip(cell, 0, (1 << bits))'),
    ('oracle/morton.py', 'order not stable',
     'perm = np.argsort(c, kind="stable")',
     'perm = np.argsort(-c.astype(np.float64), kind="quicksort")[::-1]'),
    ('oracle/lbvh.py', 'split off by one',
     '        g = lo\n',
     '        g = hi\n'),
    ('oracle/lbvh.py', 'ties not broken by index',
     'aug = [(k << 32) | i for i, k in enumerate(keys)]',
     'aug = [k << 32 for i, k in enumerate(keys)]'),
    ('oracle/rgx_oracle.c', 'bg not weighted by T',
     'rgba[4*i + 1] = r.C[1] + r.T * op->bg[1];',
     'rgba[4*i + 1] = r.C[1] + op->bg[1];'),
    ('oracle/rgx_oracle.c', 'opacity is T',
     'rgba[4*i + 3] = 1.0 - r.T;',
     'rgba[4*i + 3] = r.T;'),
    ('oracle/rgx_oracle.c', 'in-loop lattice guard dropped',
     'j = jj > j + 1 ? jj : j + 1;',
     'j = jj > j ? jj : j;'),
    ('oracle/rgx_oracle.c', 'in-loop lattice no step back',
     'int64_t jj = (int64_t)floor((th - tn) / op->dt) - 1;\n                        j = jj > j + 1 ? jj : j + 1;',
     'int64_t jj = (int64_t)floor((th - tn) / op->dt);\n                        j = jj > j + 1 ? jj : j + 1;'),
    ('oracle/rgx_oracle.c', 'samples allowed past t_f',
     'if (!(t < tf)) break;',
     'if (0) break;'),
    ('oracle/rgx_oracle.c', 'segment limit never reported',
     'if (op->max_segments > 0 && iters >= op->max_segments) { out->err = OX_ERR_ITER; break; }',
     'if (op->max_segments > 0 && iters >= op->max_segments) { break; }'),
    ('oracle/rgx_oracle.c', 'alpha from sigma without dt',
     'double e = exp(-sigma * dtk);\n            double alpha = 1.0 - e;',
     'double e = exp(-sigma * dtk);\n            double alpha = 1.0 - exp(-sigma);'),
    ('oracle/rgx_oracle.c', 'colour average not normalised',
     'double ci[3] = { S[0]/sigma, S[1]/sigma, S[2]/sigma };',
     'double ci[3] = { S[0], S[1], S[2] };'),
    ('oracle/rgx_oracle.c', 'adaptive dS one sample short',
     'dtk = a;\n                dS = ns * a;',
     'dtk = a;\n                dS = (ns - 1) * a;'),
    ('oracle/rgx_oracle.c', 'bg term of adjoint sign',
     'double dTf = a[0]*op->bg[0] + a[1]*op->bg[1] + a[2]*op->bg[2] - b;',
     'double dTf = a[0]*op->bg[0] + a[1]*op->bg[1] + a[2]*op->bg[2] + b;'),
]


def _restore_interrupted():
    if not os.path.isdir(BACKUP):
        return
    for name in os.listdir(BACKUP):
        rel = name.replace("%", os.sep)
        shutil.copy(os.path.join(BACKUP, name), os.path.join(ROOT, rel))
    shutil.rmtree(BACKUP)


def run(selection=(), timeout=120):
    """Plant each selected mutation alone; return [(label, outcome)]."""
    _restore_interrupted()
    out = []
    for path, label, before, after in MUTATIONS:
        if selection and not any(s in label for s in selection):
            continue
        src = os.path.join(ROOT, path)
        text = open(src).read()
        if text.count(before) != 1:
            out.append((label, "not applicable (source changed)"))
            continue
        os.makedirs(BACKUP, exist_ok=True)
        keep = os.path.join(BACKUP, path.replace(os.sep, "%"))
        shutil.copy(src, keep)
        try:
            with open(src, "w") as f:
                f.write(text.replace(before, after))
            try:
                r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                                   cwd=ROOT, capture_output=True, text=True, timeout=timeout)
                outcome = "caught" if r.returncode else "MISSED"
            except subprocess.TimeoutExpired:
                outcome = "timeout (the march stops advancing)"
        finally:
            shutil.copy(keep, src)
            os.remove(keep)
        out.append((label, outcome))
        print(f"{outcome:>10}  {label}", flush=True)
    _restore_interrupted()
    return out


if __name__ == "__main__":
    res = run(sys.argv[1:])
    missed = [l for l, o in res if o == "MISSED"]
    print(f"{len(res)} mutations, {len(missed)} missed" + (": " + ", ".join(missed) if missed else ""))
    sys.exit(1 if missed else 0)
