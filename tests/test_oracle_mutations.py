"""The oracle's pins against planted mistakes.  Each entry below changes one
line of the oracle the way a plausible slip would (a sign, an index, a
transposed operand, a dropped term, a clamp, a tie rule, the precision of a
decision).  A C slip is built into its own copy of the library and loaded
through ``VP_ORACLE_LIB``; a Python slip goes into a copy of the package that
shadows the real one.  The oracle's pin files then run against the copy, and
every slip must fail some pin.  The real sources are never modified."""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "vp_oracle.c")
PINS = ["test_oracle_edges.py", "test_oracle_geometry.py", "test_oracle_fk.py", "test_oracle_cost.py"]
PY_PINS = {"nn": "test_oracle_nn.py", "shortcut": "test_oracle_shortcut.py", "rrt": "test_oracle_rrt.py"}

MUTATIONS = [
 ("rodrigues sign", "(i == j ? 1.0 : 0.0) + s * K[3 * i + j]", "(i == j ? 1.0 : 0.0) - s * K[3 * i + j]"),
 ("rodrigues 1+c", "+ (1.0 - c) * K2", "+ (1.0 + c) * K2"),
 ("frame order parent/F", "        mat_mul(parent, F, PF);\n        mat_mul(PF, M", "        mat_mul(F, parent, PF);\n        mat_mul(PF, M"),
 ("frame order PF/M", "        mat_mul(PF, M, T + 16 * (j + 1));", "        mat_mul(M, PF, T + 16 * (j + 1));"),
 ("prismatic axis", "    m[3] = a[0] * d;", "    m[3] = a[1] * d;"),
 ("sphere dist +r", "    return norm3(v) - sph[3];", "    return norm3(v) + sph[3];"),
 ("capsule no upper clamp", "        if (t > 1.0) t = 1.0;\n    }\n    double v[3] = {w[0] - t * u[0], w[1] - t * u[1], w[2] - t * u[2]};\n    return", "    }\n    double v[3] = {w[0] - t * u[0], w[1] - t * u[1], w[2] - t * u[2]};\n    return"),
 ("capsule sign", "    double v[3] = {w[0] - t * u[0], w[1] - t * u[1], w[2] - t * u[2]};\n    return norm3(v) - cap[6];", "    double v[3] = {w[0] + t * u[0], w[1] + t * u[1], w[2] + t * u[2]};\n    return norm3(v) - cap[6];"),
 ("cuboid R transposed", "        double yi = R[0 * 3 + i] * d[0] + R[1 * 3 + i] * d[1] + R[2 * 3 + i] * d[2];", "        double yi = R[i * 3 + 0] * d[0] + R[i * 3 + 1] * d[1] + R[i * 3 + 2] * d[2];"),
 ("cuboid inside 0", "    return sqrt(out2) + (emax < 0.0 ? emax : 0.0);", "    return sqrt(out2);"),
 ("no self pairs", "    for (int p = 0; p < r->n_pairs; ++p) {\n        int a = r->pairs[2 * p], b = r->pairs[2 * p + 1];\n        double v[3]", "    for (int p = 0; p < 0; ++p) {\n        int a = r->pairs[2 * p], b = r->pairs[2 * p + 1];\n        double v[3]"),
 ("pair radius one side", "        double k = norm3(v) - r->sphere_radius[a] - r->sphere_radius[b];", "        double k = norm3(v) - r->sphere_radius[a];"),
 ("cuboid clearance +rs", "            double k = vpo_dist_cuboid(x, e->cuboids + 15 * o) - rs;", "            double k = vpo_dist_cuboid(x, e->cuboids + 15 * o) + rs;"),
 ("no capsules", "        for (int o = 0; o < e->n_capsules; ++o) {\n            double k = vpo_dist_capsule", "        for (int o = 0; o < 0; ++o) {\n            double k = vpo_dist_capsule"),
 ("valid strict", "    return vpo_state_clearance(r, e, q) >= 0.0;", "    return vpo_state_clearance(r, e, q) > 0.0;"),
 ("count floor", "    float steps = ceilf(dmax / res);", "    float steps = floorf(dmax / res);"),
 ("count no +1", "    int32_t k = (int32_t)steps + 1;", "    int32_t k = (int32_t)steps;"),
 ("count in double", "    float steps = ceilf(dmax / res);", "    float steps = (float)ceil((double)dmax / (double)res);"),
 ("t = i/k", "    double t = (double)i / (double)(k - 1);", "    double t = (double)i / (double)k;"),
 ("skip last state", "    for (int32_t i = 0; i < k; ++i) {\n        vpo_edge_state(q0, q1, D, k, i, q);\n        if (!vpo_state_valid", "    for (int32_t i = 0; i < k - 1; ++i) {\n        vpo_edge_state(q0, q1, D, k, i, q);\n        if (!vpo_state_valid"),
 ("classify band sign", "            if (K < -band) { cls = 1; break; }", "            if (K < band) { cls = 1; break; }"),
 ("cost pen sign grad", "                    for (int i = 0; i < 3; ++i) g[i] += -2.0 * pen * gd[i];", "                    for (int i = 0; i < 3; ++i) g[i] += 2.0 * pen * gd[i];"),
 ("cost margin dropped", "        double rs = r->sphere_radius[s] + margin;", "        double rs = r->sphere_radius[s];"),
 ("grad cuboid world rotate transposed", "    for (int i = 0; i < 3; ++i) g[i] = R[3 * i + 0] * gb[0] + R[3 * i + 1] * gb[1] + R[3 * i + 2] * gb[2];", "    for (int i = 0; i < 3; ++i) g[i] = R[0 * 3 + i] * gb[0] + R[1 * 3 + i] * gb[1] + R[2 * 3 + i] * gb[2];"),
 ("grad revolute cross sign", "                    dc[0] = a[1] * v[2] - a[2] * v[1];", "                    dc[0] = a[2] * v[1] - a[1] * v[2];"),
 ("grad axis local", "            for (int i = 0; i < 3; ++i) a[i] = JF[4 * i] * ax[0] + JF[4 * i + 1] * ax[1] + JF[4 * i + 2] * ax[2];", "            for (int i = 0; i < 3; ++i) a[i] = ax[i];"),
 ("grad origin after parent only", "            mat_mul(T + 16 * (r->parent[j] + 1), F, JF);", "            memcpy(JF, T + 16 * (r->parent[j] + 1), sizeof(JF));"),
 ("grad capsule no clamp", "        if (t > 1.0) t = 1.0;\n    }\n    double v[3] = {w[0] - t * u[0], w[1] - t * u[1], w[2] - t * u[2]};\n    double n = norm3(v);", "    }\n    double v[3] = {w[0] - t * u[0], w[1] - t * u[1], w[2] - t * u[2]};\n    double n = norm3(v);"),
 ("grad cuboid inside face sign", "        gb[imax] = y[imax] < 0.0 ? -1.0 : 1.0;", "        gb[imax] = 1.0;"),
 ("no max-steps check", "    if (!(steps <= (float)VPO_MAX_STEPS)) return -1;\n", ""),
 ("no minimum of 2", "    return k < 2 ? 2 : k;", "    return k;"),
 ("explicit count unbounded", "    if (k < 2 || k > VPO_MAX_STEPS + 1 || !endpoints_finite(q0, q1, D)) return 0;", "    if (k < 2 || !endpoints_finite(q0, q1, D)) return 0;"),
 ("classify count unbounded", "    if (k < 2 || k > VPO_MAX_STEPS + 1 || !endpoints_finite(q0, q1, D)) {", "    if (k < 2 || !endpoints_finite(q0, q1, D)) {"),
 ("edge k<2 accepted", "    if (k < 2 || k > VPO_MAX_STEPS + 1 || !endpoints_finite(q0, q1, D)) return 0;", "    if (k > VPO_MAX_STEPS + 1 || !endpoints_finite(q0, q1, D)) return 0;"),
 ("non-finite state not invalid", "    if (!all_finite(q, r->n_joints)) return -INFINITY;\n", ""),
 ("non-finite endpoint count", "        if (!isfinite(q0[d]) || !isfinite(q1[d])) return -1;\n", ""),
 ("edge state from q1", "    for (int d = 0; d < D; ++d) q[d] = (double)q0[d] + t * ((double)q1[d] - (double)q0[d]);", "    for (int d = 0; d < D; ++d) q[d] = (double)q1[d] + t * ((double)q0[d] - (double)q1[d]);"),
]


def _caught(tmp, idx, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {name!r} no longer matches the source"
    path = os.path.join(tmp, f"m{idx}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp, f"m{idx}.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-I", os.path.dirname(SRC), "-o", lib, path, "-lm"])
    env = dict(os.environ, VP_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
                       + [os.path.join(HERE, p) for p in PINS], cwd=ROOT, env=env, capture_output=True, text=True)
    return r.returncode == 1  # 1: some test failed (not a collection or usage error)


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            caught = list(ex.map(lambda a: _caught(tmp, *a), [(i, *m) for i, m in enumerate(MUTATIONS)]))
    survivors = [m[0] for m, c in zip(MUTATIONS, caught) if not c]
    assert not survivors, f"no pin catches: {survivors}"


PY_MUTATIONS = [
 ("nn", "l1 distance", '        d = np.einsum("nmd,nmd->nm", diff, diff)', '        d = np.abs(diff).sum(axis=2)'),
 ("nn", "ties to the highest index", "        i = np.argmin(d, axis=1)  # first minimum: the lowest index on ties", "        i = d.shape[1] - 1 - np.argmin(d[:, ::-1], axis=1)"),
 ("nn", "second best not excluded", "            d[np.arange(b - a), i] = np.inf\n", ""),
 ("shortcut", "round not floor", "    i = min(int(np.floor(np.float32(u0) * nf)), n - 1)", "    i = min(int(np.round(np.float32(u0) * nf)), n - 1)"),
 ("shortcut", "no clamp", "    j = min(int(np.floor(np.float32(u1) * nf)), n - 1)", "    j = int(np.floor(np.float32(u1) * nf))"),
 ("shortcut", "no swap", "    if i > j:\n        i, j = j, i\n", ""),
 ("shortcut", "adjacent allowed", "    return (i, j) if j - i >= 2 else None", "    return (i, j) if j - i >= 1 else None"),
 ("shortcut", "product in float64", "    i = min(int(np.floor(np.float32(u0) * nf)), n - 1)", "    i = min(int(np.floor(float(u0) * n)), n - 1)"),
 ("shortcut", "splice off by one", "                paths[p, i + 1:i + 1 + (n - j)] = paths[p, j:n].copy()", "                paths[p, i:i + (n - j)] = paths[p, j:n].copy()"),
 ("shortcut", "length off by one", "                lengths[p] = n - (j - i - 1)", "                lengths[p] = n - (j - i)"),
 ("rrt", "ties to the highest index", "    i = int(np.argmin(acc))", "    i = int(n - 1 - np.argmin(acc[::-1]))"),
 ("rrt", "reach strict", "    if dist <= F(rng):", "    if dist < F(rng):"),
 ("rrt", "steer from q", "    return near + s * (q - near), ADVANCED", "    return q + s * (near - q), ADVANCED"),
 ("rrt", "no duplicate check", "    if d2 == F(0):\n        return REACHED, i\n", ""),
 ("rrt", "trees never swap", "        a = 1 - a\n    return 0", "    return 0"),
 ("rrt", "meeting node twice", "                    path = pa[::-1] + pb[1:]           # start ... meet ... goal", "                    path = pa[::-1] + pb           # start ... meet ... goal"),
 ("rrt", "iterations off by one", "                return 1, it + 1, np.array", "                return 1, it, np.array"),
 ("rrt", "steer in float64", "    return near + s * (q - near), ADVANCED", "    return (near.astype(np.float64) + float(s) * (q.astype(np.float64) - near)).astype(F), ADVANCED"),
 ("rrt", "nearest in float64", "        acc = acc + t[:, d] * t[:, d]     # product, then sum, each rounded", "        acc = (acc.astype(np.float64) + t[:, d].astype(np.float64) ** 2).astype(F)"),
 ("rrt", "path orientation when B moved first", "                    path = pb[::-1] + pa[1:]", "                    path = pa[::-1] + pb[1:]"),
 ("rrt", "goal validity ignored", "    if np.any(k < 0):", "    if k[0] < 0:"),
 ("rrt", "no capacity check", "    if tree.n == tree.nodes.shape[0]:\n        return TRAPPED, -1\n", ""),
 ("rrt", "band never flagged", "    band = [bool(np.any(np.abs(k) <= 1e-4))]", "    band = [False]"),
 ("shortcut", "band on collisions", "            band[p] |= c == 2", "            band[p] |= c == 1"),
 ("nn", "distance of the wrong row", "        d1[a:b] = d[np.arange(b - a), i]", "        d1[a:b] = d[0, i]"),
 ("nn", "second best from the first row", "            d2[a:b] = d.min(axis=1)", "            d2[a:b] = d[0].min()"),
]


def _py_caught(tmp, idx, mod, name, old, new):
    import oracle
    root = os.path.join(tmp, f"p{idx}")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(root, "oracle"),
                    ignore=shutil.ignore_patterns("*.so", "*.so.*", "__pycache__"))
    f = os.path.join(root, "oracle", mod + ".py")
    src = open(f).read()
    assert src.count(old) == 1, f"mutation {name!r} no longer matches oracle/{mod}.py"
    with open(f, "w") as fh:
        fh.write(src.replace(old, new))
    env = dict(os.environ, VP_ORACLE_LIB=oracle.build(), PYTHONPATH=root + os.pathsep + ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        os.path.join(HERE, PY_PINS[mod])], cwd=root, env=env, capture_output=True, text=True)
    return r.returncode == 1


def test_every_planted_mistake_in_the_python_oracles_fails_a_pin():
    import oracle
    oracle.build()
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            caught = list(ex.map(lambda a: _py_caught(tmp, *a), [(i, *m) for i, m in enumerate(PY_MUTATIONS)]))
    survivors = [f"{m[0]}: {m[1]}" for m, c in zip(PY_MUTATIONS, caught) if not c]
    assert not survivors, f"no pin catches: {survivors}"
