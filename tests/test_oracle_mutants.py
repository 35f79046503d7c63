"""The oracle's pins catch plausible mistakes: each case below plants one
mistake (a dropped term, a wrong sign, constant, exponent or index, a
transposed operand, an unstable order, ...) in a copy of the oracle, on the
CPU, and the oracle pins (tests/test_oracle_*.py) must then fail.  A clean
copy must pass them, so the harness itself is checked too.  Every mutant
here changes what the oracle computes (none is an equivalent rewrite)."""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_grid.py", "tests/test_oracle_drag.py", "tests/test_oracle_implicit.py",
        "tests/test_oracle_map.py", "tests/test_oracle_mlp.py"]
C = "oracle/cg_oracle.c"
PY = "oracle/mlp.py"

# (file, text in the oracle, planted replacement, what the mistake is)
MUTANTS = [
    (C, 'static double sphere_volume(double d) { return M_PI * d * d * d / 6.0; }',
     'static double sphere_volume(double d) { return M_PI * d * d * d / 8.0; }',
     'sphere volume constant'),
    (C, '        eps[c] = 1.0 - ph;',
     '        eps[c] = ph;',
     'porosity as solid fraction'),
    (C, '    return idx[0] + g.nb[0] * (idx[1] + g.nb[1] * idx[2]);',
     '    return idx[2] + g.nb[2] * (idx[1] + g.nb[1] * idx[0]);',
     'transposed linear cell index'),
    (C, '        if (!(q >= 0.0 && q <= (double)g.nb[a])) out = 1;',
     '        if (!(q >= 0.0 && q < (double)g.nb[a])) out = 1;',
     'upper domain face counted outside'),
    (C, '    for (int64_t p = 0; p < n; ++p) perm[cursor[cell[p]]++] = (int32_t)p;',
     '    for (int64_t p = n - 1; p >= 0; --p) perm[cursor[cell[p]]++] = (int32_t)p;',
     'unstable (reversed) order within a cell'),
    (C, '            mean[comp] = ks_get(&k) / cnt;',
     '            mean[comp] = ks_get(&k) / (cnt - 1.0);',
     'mean over r^3 - 1'),
    (C, '            var_bulk[cb] = ks_get(&k) / cnt;',
     '            var_bulk[cb] = ks_get(&k) / (cnt - 1.0);',
     'sample variance'),
    (C, '                int64_t f = (I * r + di) + nxf * ((J * r + dj) + nyf * (int64_t)(K * r + dk));\n                ks_add(&k, u_fine[comp * g.nfine + f]);',
     '                int64_t f = (I * r + di) + nxf * ((J + dj) + nyf * (int64_t)(K * r + dk));\n                ks_add(&k, u_fine[comp * g.nfine + f]);',
     'averaging: bulk row J not scaled by r'),
    (C, '        double xi = (x[a] - G->x0[a]) / g.H[a] - 0.5;',
     '        double xi = (x[a] - G->x0[a]) / g.H[a];',
     'stencil from cell corners, not centres'),
    (C, '        else if (tt > 1.0) { tt = 1.0; cl = 1; }',
     '        else if (tt > 1.0) { cl = 1; }',
     'linear extrapolation in the outer half cell'),
    (C, '            double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);',
     '            double w = (dx ? 1.0 - t[0] : t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);',
     'flipped x weights'),
    (C, '                    if (b == a) w *= d3[b] ? 1.0 : -1.0;',
     '                    if (b == a) w *= d3[b] ? -1.0 : 1.0;',
     'gradient sign'),
    (C, '            acc /= g.H[a];',
     '            acc *= g.H[a];',
     'gradient scaled by H, not 1/H'),
    (C, '        double cd_s = 0.63 * sqrt(smag) + 4.8 * sqrt(mu / (rho * eps * d));',
     '        double cd_s = 0.63 * sqrt(smag) + 4.8 * sqrt(mu / (rho * d));',
     'Di Felice Re without eps'),
    (C, '            double l = 1.5 - log10(Re);',
     '            double l = 1.5 - log(Re);',
     'natural log in the exponent'),
    (C, '            chi = 3.7 - 0.65 * exp(-l * l / 2.0);',
     '            chi = 3.7 + 0.65 * exp(-l * l / 2.0);',
     'exponent sign'),
    (C, '(M_PI * d * d / 4.0) * eps * eps * pow(eps, -chi);',
     '(M_PI * d * d / 4.0) * eps * pow(eps, -chi);',
     'dropped eps factor'),
    (C, '            return (150.0 * phi * mu / (eps * d * d) + 1.75 * rho * smag / d) * vp;',
     '            return (150.0 * phi * phi * mu / (eps * d * d) + 1.75 * rho * smag / d) * vp;',
     'Ergun (1-eps) not cancelled'),
    (C, '            return (150.0 * phi * mu / (eps * d * d) + 1.75 * rho * smag / d) * vp;',
     '            return (150.0 * phi * mu / (eps * d * d) + 1.75 * rho * smag * smag / d) * vp;',
     'Ergun inertial term squared'),
    (C, '        if (eps < G->eps_switch) {',
     '        if (eps <= G->eps_switch) {',
     'switch tie to Ergun'),
    (C, '            return 0.75 * cd_s * eps * rho * pow(eps, -2.65) / d * vp;',
     '            return 0.75 * cd_s * eps * rho * pow(eps, -1.65) / d * vp;',
     'Wen-Yu exponent'),
    (C, '(1.0 + 0.15 * pow(eRe, 0.687));',
     '(1.0 + 0.15 * pow(Re, 0.687));',
     'Wen-Yu correction at Re, not eps Re'),
    (C, '            else cd_s = 0.44 * smag;',
     '            else cd_s = 0.44;',
     'Newton regime without |s|'),
    (C, '    if (eps < G->eps_min) { eps = G->eps_min; cl = 1; }',
     '    if (eps < G->eps_min) { cl = 1; }',
     'eps_min counted, not applied'),
    (C, '            S_bulk[comp * g.nbulk + c] = -ks_get(&k) / g.VB;',
     '            S_bulk[comp * g.nbulk + c] = ks_get(&k) / g.VB;',
     'reaction sign'),
    (C, '        double x[3] = {G->x0[0] + (i + 0.5) * g.h[0],',
     '        double x[3] = {G->x0[0] + i * g.h[0],',
     'projection at fine nodes'),
    (C, '            double x = pos_d[4 * p + a] + dt * u;',
     '            double x = pos_d[4 * p + a] + dt * vel[4 * p + a];',
     'position-first Euler'),
    (C, '        double m = G->rho_p * sphere_volume(pos_d[4 * p + 3]);\n        for (int a = 0; a < 3; ++a) {\n            double u',
     '        double m = G->rho_f * sphere_volume(pos_d[4 * p + 3]);\n        for (int a = 0; a < 3; ++a) {\n            double u',
     'fluid density as particle mass'),
    (C, '            if (x < lo) { x = 2.0 * lo - x; u = -u; }',
     '            if (x < lo) { x = 2.0 * lo - x; }',
     'wall without velocity reversal'),
    (C, '            for (int a = 0; a < 3; ++a) ks_add(&k[1 + a], beta * vel[4 * p + a]);',
     '            for (int a = 0; a < 3; ++a) ks_add(&k[1 + a], beta * uf[a]);',
     'explicit part with the fluid velocity'),
    (C, '    return hi > lo ? hi - lo : 0.0;',
     '    return hi - lo;',
     'negative overlaps'),
    (C, '        for (int c = 0; c < ncomp; ++c) s_fine[c * nfn + cf] = ks_get(&acc[c]) / Vf;',
     '        for (int c = 0; c < ncomp; ++c) s_fine[c * nfn + cf] = ks_get(&acc[c]);',
     'projection without 1/V_f'),
    (C, '        for (int c = 0; c < ncomp; ++c) u_bulk[c * nbk + cb] = W > 0.0 ? ks_get(&acc[c]) / W : 0.0;',
     '        for (int c = 0; c < ncomp; ++c) u_bulk[c * nbk + cb] = W > 0.0 ? ks_get(&acc[c]) / W : 1.0;',
     'uncovered cells not zero'),
    (C, '    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;',
     '    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) - x;',
     'compensation term sign'),
    (PY, '    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))',
     '    return 0.5 * x * (1.0 + erf(x / 2.0))',
     'GELU scale'),
    (PY, '    return cdf + x * pdf',
     '    return cdf',
     'GELU derivative without x pdf'),
    (PY, '    dA1 = q(dZ2) @ q(p["W2"]).T',
     '    dA1 = q(dZ2) @ q(p["W2"])',
     'transposed W2 in backprop'),
    (PY, '    g["b2"] = dZ2.sum(axis=0)',
     '    g["b2"] = dZ2.mean(axis=0)',
     'bias gradient as a mean'),
    (PY, '    dc = 2.0 * r / B',
     '    dc = r / B',
     'loss gradient factor'),
    (PY, '        mh = M[k] / (1 - b1 ** t)',
     '        mh = M[k]',
     'Adam without bias correction'),
    (PY, '    r = ((u + 0x7FFF + lsb) >> 16) << 16',
     '    r = (u >> 16) << 16',
     'bf16 by truncation'),
    (C, '        f[1] = log10(1.0 + Re);',
     '        f[1] = log10(Re + 1e-300);',
     'feature log10 Re, not log10(1 + Re)'),
    (C, '        target[p] = nn > 0.0 ? dot / nn : 1.0;',
     '        target[p] = nn > 0.0 ? dot / sqrt(nn) : 1.0;',
     'target normalised by |F_stale|'),
    (C, '        for (int comp = 0; comp < 4; ++comp) coef[comp * g.nbulk + c] = ks_get(&k[comp]) / g.VB;',
     '        for (int comp = 0; comp < 4; ++comp) coef[comp * g.nbulk + c] = ks_get(&k[comp]);',
     'coefficients without 1/V_B'),
    (C, '            ks_add(&k[1], (1.0 - eps_bulk[c]) * g.VB);',
     '            ks_add(&k[1], (1.0 - eps_bulk[c]) * g.Vf);',
     'deposited volume sum with V_f'),
    (C, '    if (G->interp == 1) {',
     '    if (G->interp == 2) {',
     'cell-value mode ignored'),
]


def _run(mutant):
    """Copy the oracle, the input generators and the pins to a scratch
    folder, plant the mistake (None: none) and run the pins there."""
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        skip = shutil.ignore_patterns("_build", "__pycache__")
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"), ignore=skip)
        shutil.copytree(os.path.join(ROOT, "synth"), os.path.join(d, "synth"), ignore=skip)
        os.makedirs(os.path.join(d, "tests"))
        shutil.copy(os.path.join(ROOT, "tests", "conftest.py"), os.path.join(d, "tests"))
        shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
        for p in PINS:
            shutil.copy(os.path.join(ROOT, p), os.path.join(d, "tests"))
        if mutant is not None:
            f, old, new, _ = mutant
            path = os.path.join(d, f)
            src = open(path).read()
            if src.count(old) != 1:
                return "text to replace found %d times" % src.count(old)
            open(path, "w").write(src.replace(old, new))
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS, cwd=d,
                           capture_output=True, text=True, timeout=600)
        failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED tests/test_oracle_")]
        return (r.returncode, failed[0] if failed else r.stdout[-300:])
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_clean_copy_passes_and_every_mutant_is_caught():
    assert _run(None)[0] == 0
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(_run, MUTANTS))
    survivors = [(m[3], res) for m, res in zip(MUTANTS, results)
                 if not (isinstance(res, tuple) and res[0] == 1 and res[1].startswith("FAILED"))]
    assert not survivors, survivors
