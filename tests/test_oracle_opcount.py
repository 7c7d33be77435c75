"""The operation count of the oracle, pinned to the paper's algorithms as
written: the oracle's source compiled with an op-counting scalar type
(oracle/opcount.cpp) must perform exactly the operations the printed
algorithms contain, one rounded operation per operator.

Counted by hand from the algorithms:
  Algorithm 1, I1 = (A00 + A11) + A22: 2 additions.
  Algorithm 2: d0, d1, d2 (3 subtractions); offdiag = A01 A10 + A02 A20 +
    A12 A21 (3 products, 2 sums); diag = (d0^2 + d1^2 + d2^2)/6 (3 products,
    2 sums, 1 division); diag + offdiag (1 sum): 8 add, 6 mul, 1 div.
  Algorithm 4: d's (3), t1 = d1 + d2, t2 = d0 - d2, t3 = -d0 - d1 (3 and one
    negation); offdiag = A01 A12 A20 + A02 A10 A21 (4 products, 1 sum); mixed
    = (A01 A10 t1 + A02 A20 t2 + A12 A21 t3)/3 (6 products, 2 sums, 1
    division); t1 t2 t3 / 27 (2 products, 1 division); (offdiag + mixed) -
    diag (2): 11 add, 12 mul, 2 div, 1 neg.
  Algorithm 5: d's (3); dx(M) has r1 with two triple products (4 mul, 1
    add), r2..r7 with three (6 mul, 2 add each; r2 and r7 lead with a
    negated factor), r8..r14 with four (8 mul, 3 add each; r12 leads with a
    negation): 96 mul, 34 add, 3 neg, done for A and A^T; sum_i w_i u_i v_i
    (2 products and 1 sum per term, 14 terms): 85 add, 220 mul, 6 neg.
  Algorithm 6: the clamps of J2 and Delta (2 comparisons); sqrt(27 Delta),
    27 J3, atan2; 2 sqrt(3 J2); for k = 1, 2, 3: (phi + 2 pi k)/3, its
    cosine, I1 + rad cos, /3: 10 mul, 6 add, 6 div, 2 sqrt, 1 atan2, 3 cos.
A dropped or added term anywhere changes these numbers."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W

ZERO = dict(add=0, mul=0, div=0, neg=0, sqrt=0, atan2=0, cos=0, cmp=0, abs=0)
EXPECTED = {
    "I1": dict(ZERO, add=2),
    "J2": dict(ZERO, add=8, mul=6, div=1),
    "J3": dict(ZERO, add=11, mul=12, div=2, neg=1),
    "Delta": dict(ZERO, add=85, mul=220, neg=6),
    "eigvals_from_invariants": dict(ZERO, add=6, mul=10, div=6, sqrt=2, atan2=1, cos=3, cmp=2),
}


def total(*names):
    out = dict(ZERO)
    for n in names:
        for k, v in EXPECTED[n].items():
            out[k] += v
    return out


EXPECTED["invariants"] = total("I1", "J2", "J3", "Delta")
EXPECTED["eigvals"] = total("I1", "J2", "J3", "Delta", "eigvals_from_invariants")


@pytest.mark.parametrize("fn", sorted(EXPECTED))
def test_counts_are_the_printed_algorithms(fn):
    A = W.workload2(n=3, device="cpu", seed=77).A.numpy()
    for a in A:
        arg = oracle.invariants(a[None])[0] if fn == "eigvals_from_invariants" else a
        counts, _ = oracle.opcount(fn, arg)
        assert counts == EXPECTED[fn], (fn, counts)


def test_the_bench_quotes_the_pinned_count():
    import bench
    e = EXPECTED["eigvals"]
    assert bench.ORACLE_OPS_EIGVALS_GENERAL9 == {k: e[k] for k in
                                                 ("add", "mul", "div", "neg", "sqrt", "atan2",
                                                  "cos")}


def test_counted_run_computes_the_oracle():
    """The counting type carries the oracle's binary64 values unchanged."""
    A = W.workload2(n=16, device="cpu", seed=78).A.numpy()
    lam = oracle.eigvals(A)
    inv = oracle.invariants(A)
    for i, a in enumerate(A):
        assert np.array_equal(oracle.opcount("eigvals", a)[1], lam[i])
        assert np.array_equal(oracle.opcount("invariants", a)[1], inv[i])


def test_a_dropped_term_changes_the_count(tmp_path):
    """Plant a slip in a copy of the oracle (r8 of Algorithm 5 without its
    last term) and count again: the pin above would fail."""
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "eig3_oracle.c")).read()
    line = "r[7] = ((M12 * d0 * d1 - M02 * M10 * d1) + M01 * M10 * M12) - M12 * M12 * M21;"
    assert line in src
    (tmp_path / "eig3_oracle.c").write_text(
        src.replace(line, "r[7] = (M12 * d0 * d1 - M02 * M10 * d1) + M01 * M10 * M12;"))
    shutil.copy(os.path.join(here, "opcount.cpp"), tmp_path / "opcount.cpp")
    so = tmp_path / "libopc.so"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c++17",
                    "-I", str(tmp_path), "-o", str(so), str(tmp_path / "opcount.cpp"),
                    "-lpthread"], check=True)
    import ctypes
    lib = ctypes.CDLL(str(so))
    a = W.workload2(n=1, device="cpu", seed=79).A.numpy()[0].copy()
    counts = np.zeros(9, dtype=np.int64)
    res = np.zeros(4)
    assert lib.eig3o_opcount(5, a.ctypes.data, counts.ctypes.data, res.ctypes.data) == 0
    assert (int(counts[0]), int(counts[1])) == (85 - 2, 220 - 4)   # one term of dx(A), dx(A^T)
