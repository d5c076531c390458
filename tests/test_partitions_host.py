"""Host-side check of the order-p contraction kernel's compile-time term table
(paper_1506_04448_gb300/csrc/partitions.h, plain constexpr C++): compiled with the host C++
compiler and compared term by term with the table the order-p oracle's definitions give
(partitions of p, z_lambda; readings 24-28 of the order-p sketches).  No GPU needed."""
import os
import shutil
import subprocess
from collections import Counter

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1506_04448_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "partitions.h"
template <int P> void dump() {
  constexpr tsk::CTerms<P> t = tsk::TermTable<P>::value;
  for (int q = 0; q < t.count; ++q) {
    std::printf("%d %d %.9g", P, t.target[q], (double)t.coef[q]);
    for (int j = 0; j < t.nparts[q]; ++j) std::printf(" %d", t.parts[q][j]);
    std::printf("\n");
  }
}
int main() { dump<3>(); dump<4>(); dump<5>(); dump<6>(); return 0; }
"""


def expected_terms(p):
    """The term multiset of the estimators: (0, 1/z, lambda) for lambda != (p); (k, m_k/z,
    lambda minus one k) for every part size k < p of lambda."""
    out = []
    for lam in O.orderp.partitions(p):
        z = O.orderp.z_of(lam)
        if lam != (p,):
            out.append((0, 1.0 / z, tuple(sorted(lam))))
        for k, mk in Counter(lam).items():
            if k < p:
                rest = list(lam)
                rest.remove(k)
                out.append((k, mk / z, tuple(sorted(rest))))
    return out


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("partitions")
    src, exe = d / "dump.cpp", d / "dump"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    rows = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for row in rows:
        if row.strip():
            f = row.split()
            got.setdefault(int(f[0]), []).append((int(f[1]), float(f[2]), tuple(sorted(int(x) for x in f[3:]))))
    return got


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_compile_time_term_table_matches_the_partition_expansion(table, p):
    got = sorted(table[p])
    want = sorted(expected_terms(p))
    assert len(got) == len(want)
    for (tg, cg, pg), (tw, cw, pw) in zip(got, want):
        assert (tg, pg) == (tw, pw)
        assert cg == pytest.approx(cw, rel=1e-7)


def test_order3_table_is_app_b():
    """p = 3: Y = s1^3/6 + s2 s1/2 (+ s3/3 read directly), F R_1 = s1^2/2 + s2/2, F R_2 = s1/2."""
    want = {(0, (1, 1, 1)): 1 / 6, (0, (1, 2)): 1 / 2, (1, (1, 1)): 1 / 2, (1, (2,)): 1 / 2,
            (2, (1,)): 1 / 2}
    assert len(expected_terms(3)) == len(want)
    for tg, c, parts in expected_terms(3):
        assert want[(tg, parts)] == pytest.approx(c)
