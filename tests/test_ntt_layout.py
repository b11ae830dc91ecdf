"""Host-side checks of the register / shared-memory layouts of the block NTT (csrc/ntt.cuh):
the header's layout functions are compiled for the CPU with nvcc and exercised for every pass
of N = 2^10 .. 2^14 with 8 and 16 residues per thread. Checked: every pass layout is a
bijection of (thread, register) onto the N indices; it splits into a per-thread base and a
per-register offset on disjoint bits (the kernels add them); the XOR-swizzled shared-memory
slots of one register across a half-warp fall in 16 distinct 8-byte banks (no conflicts); and
exchange_in_warp(), which lets an exchange use a warp barrier instead of a block barrier, is
true exactly when every warp holds the same indices in both layouts. Both forms of a partial
last pass are checked: warp-adjacent groups (the unrolled transforms) and groups strided by the
thread count (the compact transforms)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_03568_gb300", "csrc")

CHECK = r'''
#include "ntt.cuh"
#include <algorithm>
#include <cstdio>
#include <vector>
using namespace ichee;
template <int E>
static int check(int logn)
{
    const int le = E == 16 ? 4 : 3, n = 1 << logn, T = n / E;
    int bad = 0;
    std::vector<int> passes;
    for (int s0 = 0; s0 < logn; s0 += le) passes.push_back(s0);
    for (int wt = 0; wt < 2; ++wt)
    for (int s0 : passes) {
        std::vector<int> seen(n, 0);
        for (int t = 0; t < T; ++t)
            for (int e = 0; e < E; ++e) {
                const int x = elem_index_of(logn, s0, E, t, e, wt);
                const int xb = elem_index_of(logn, s0, E, t, 0, wt), xo = elem_index_of(logn, s0, E, 0, e, wt);
                if (x < 0 || x >= n || seen[x]++) ++bad;
                if (x != (xb | xo) || (xb & xo)) ++bad;
            }
        for (int e = 0; e < E; ++e)
            for (int w = 0; w < T; w += 16) {
                int cnt[16] = {0};
                for (int t = w; t < w + 16; ++t)
                    if (++cnt[swz<E>(elem_index_of(logn, s0, E, t, e, wt)) & 15] > 1) ++bad;
            }
    }
    for (size_t i = 0; i + 1 < passes.size(); ++i) {
        bool same = true;
        for (int w = 0; w < T && same; w += 32) {
            std::vector<int> a, b;
            for (int t = w; t < w + 32; ++t)
                for (int e = 0; e < E; ++e) {
                    a.push_back(elem_index_of(logn, passes[i], E, t, e));
                    b.push_back(elem_index_of(logn, passes[i + 1], E, t, e));
                }
            std::sort(a.begin(), a.end());
            std::sort(b.begin(), b.end());
            same = a == b;
        }
        if (same != exchange_in_warp(logn, passes[i], passes[i + 1], E)) ++bad;
        printf("%d %d %d %d %d\n", E, logn, passes[i], passes[i + 1], (int)same);
    }
    return bad;
}
int main()
{
    int bad = 0;
    for (int logn = 10; logn <= 14; ++logn) bad += check<8>(logn) + check<16>(logn);
    printf("bad %d\n", bad);
    return bad != 0;
}
'''


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_ntt_layouts(tmp_path):
    cc = nvcc()
    if cc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "layout_check.cu"
    src.write_text(CHECK)
    exe = tmp_path / "layout_check"
    r = subprocess.run([cc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    rows = [tuple(int(v) for v in line.split()) for line in r.stdout.splitlines() if not line.startswith("bad")]
    in_warp = {(E, logn, a, b) for E, logn, a, b, same in rows if same}
    # the exchanges the N = 8192 kernels with 8 residues per thread (1024 threads) run with a
    # warp barrier: the last two of each transform
    assert (8, 13, 6, 9) in in_warp and (8, 13, 9, 12) in in_warp
    assert (8, 13, 0, 3) not in in_warp and (8, 13, 3, 6) not in in_warp
