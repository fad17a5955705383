"""The boundary is a C ABI: a plain C99 program that includes
include/pmlbie.h (no C++ and no CUDA headers), links libpmlbie.so, builds a
problem's host tables and reads them back, then checks a parameter error.
Its output must equal what the Python binding reads from the same library.
No GPU: creation and the host accessors never touch a device."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <string.h>
#include "pmlbie.h"

int main(void) {
    pmlbie_params p;
    memset(&p, 0, sizeof p);
    p.struct_size = sizeof p;
    p.k1 = 12.566370614359172; p.k2 = 18.84955592153876;
    p.a1 = 2.5; p.T = 1.0; p.S = 3.0; p.p = 6; p.N = 96; p.M = 32;
    p.curve_kind = PMLBIE_CURVE_GAUSS_BUMP;
    p.bump_h = 0.2; p.bump_w = 0.5; p.bump_R = 1.0;
    p.taylor_L = 5; p.split_c = 8.0;
    p.wavy_R = 1.0; p.wavy_eps = 0.1; p.wavy_m = 3;
    pmlbie_problem* prob = NULL;
    if (pmlbie_create(&p, &prob) != PMLBIE_OK) { printf("create failed: %s\n", pmlbie_last_error()); return 1; }
    double rho[96], z[96], sp[96], t[96], Da[96], Db[96];
    if (pmlbie_nodes(prob, rho, z, sp, t, 96) != PMLBIE_OK) return 2;
    if (pmlbie_diagonal(prob, Da, Db, 96) != PMLBIE_OK) return 3;
    int ng = 0, nc = 0;
    if (pmlbie_near_count(prob, &ng, &nc) != PMLBIE_OK) return 4;
    printf("%d %d\n", ng, nc);
    for (int i = 0; i < 96; ++i) printf("%.17g %.17g %.17g\n", rho[i], z[i], Da[i]);
    int rc = pmlbie_nodes(prob, rho, z, sp, t, 95);          /* wrong length */
    printf("%d\n", rc == PMLBIE_EINVAL);
    pmlbie_destroy(prob);
    p.M = 30;                                                /* 4 does not divide M */
    prob = NULL;
    printf("%d %d\n", pmlbie_create(&p, &prob) == PMLBIE_EINVAL, prob == NULL);
    return 0;
}
"""


def test_plain_c_consumer(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2412_11162_gb300 import Problem
    from paper_2412_11162_gb300 import binding as B
    src = tmp_path / "consumer.c"
    src.write_text(C_SRC)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(B.LIB_PATH)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-lpmlbie", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    cuda_lib = "/usr/local/cuda/lib64"
    env["LD_LIBRARY_PATH"] = cuda_lib + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.split("\n")
    ng, nc = map(int, lines[0].split())
    vals = np.array([[float(v) for v in ln.split()] for ln in lines[1:97]])
    assert lines[97] == "1" and lines[98] == "1 1"
    P = Problem(4 * np.pi, 6 * np.pi, 96, 32)
    nd = P.nodes()
    Da, _ = P.diagonal()
    assert P.near_count() == (ng, nc)
    P.close()
    assert np.array_equal(vals[:, 0], nd["rho"]) and np.array_equal(vals[:, 1], nd["z"])
    assert np.array_equal(vals[:, 2], Da)
