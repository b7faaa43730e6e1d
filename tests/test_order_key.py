"""The slab exchange decides owners and ghosts by unsigned comparisons of order keys of
FP64 coordinates and boundaries (dem_halo.h). Pin: for every pair of non-NaN doubles,
a < b and a <= b agree with the comparisons of their keys (-0 equals +0; infinities,
subnormals, random bit patterns), and the boundary keys are the keys of the FP64
differences and sums. Host code only: the header's host path, compiled by nvcc here."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>
#include <vector>
#include "dem_halo.h"
using namespace demgb;

static int check(double a, double b) {
    const uint64_t ka = order_key(a), kb = order_key(b);
    return ((a < b) != (ka < kb)) + ((a <= b) != (ka <= kb)) + ((a == b) != (ka == kb));
}

int main() {
    const double inf = std::numeric_limits<double>::infinity();
    const double tiny = std::numeric_limits<double>::denorm_min();
    std::vector<double> sp = {0.0, -0.0, tiny, -tiny, DBL_MIN, -DBL_MIN, 1e-310, -1e-310, 1.0, -1.0,
                              std::nextafter(1.0, 2.0), std::nextafter(1.0, 0.0), -std::nextafter(1.0, 2.0),
                              DBL_MAX, -DBL_MAX, inf, -inf, 0.05, -0.05, 0.0505, -0.0505};
    long bad = 0, n = 0;
    for (double a : sp)
        for (double b : sp) { bad += check(a, b); ++n; }
    std::mt19937_64 rng(12345);
    std::uniform_real_distribution<double> u(-0.06, 0.06);
    for (int i = 0; i < 400000; ++i) {
        uint64_t x = rng(), y = rng();
        double a, b;
        std::memcpy(&a, &x, 8);
        std::memcpy(&b, &y, 8);
        if (!std::isnan(a) && !std::isnan(b)) { bad += check(a, b); ++n; }
        const double c = u(rng);
        const double d = (i & 1) ? std::nextafter(c, inf) : u(rng);   // neighbours and random pairs
        bad += check(c, d) + check(d, c) + check(c, c);
        n += 3;
    }
    HaloGeom g{};
    g.nslabs = 3;
    g.zb[0] = -inf; g.zb[1] = -0.0123456789; g.zb[2] = 0.0314159; g.zb[3] = inf;
    g.G = 2.2e-3;
    set_keys(g);
    for (int t = 0; t <= 3; ++t) bad += g.kb[t] != order_key(g.zb[t]);
    for (int t = 0; t < 3; ++t) bad += (g.klo[t] != order_key(g.zb[t] - g.G)) + (g.khi[t] != order_key(g.zb[t + 1] + g.G));
    std::printf("%ld %ld\n", bad, n);
    return bad != 0;
}
'''


def test_order_keys_compare_like_doubles(tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    src = tmp_path / "order_key_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "order_key_check"
    csrc = os.path.join(ROOT, "paper_1301_1714_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"), "-I" + csrc, str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    bad, n = (int(k) for k in out.stdout.split())
    assert n > 1_000_000
    assert bad == 0 and out.returncode == 0
