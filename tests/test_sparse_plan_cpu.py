"""The compile-time plan of the sparse LU the Rosenbrock kernels use on the large stiff models
(Appendix: HIRES, POLLU), checked on the host: a small program built with nvcc prints the plan
the kernels are compiled with (elimination order, filled pattern, operation lists), and

* the order is the greedy minimum-degree order of the symmetrised Jacobian pattern (fewest
  remaining neighbours first, ties to the lower index), recomputed here from the oracle's
  Jacobians;
* the filled pattern is the symbolic elimination of the permuted pattern, recomputed here;
* executing the printed operation lists in NumPy on W = I - hg J (the oracle's Jacobian at a
  random state) reproduces the LU factors of P W P^T and solves W x = b to round-off, and the
  pivot checks in the list cover every entry below each pivot.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_06835_gb300", "csrc")

DUMP = r"""
#include <cstdio>
#include "ens_device.cuh"
template <class RHS> void dump(const char* name) {
  constexpr auto& P = ens::SpPlanOf<RHS>::plan;
  printf("model %s %d %d\n", name, RHS::D, P.nnz);
  printf("order");
  for (int k = 0; k < RHS::D; ++k) printf(" %d", P.order[k]);
  printf("\n");
  for (int r = 0; r < RHS::D; ++r) {
    printf("slot");
    for (int c = 0; c < RHS::D; ++c) printf(" %d", P.slot[r][c]);
    printf("\n");
  }
  for (int i = 0; i < P.nfac; ++i)
    printf("fac %d %d %d %d\n", P.fac[i].kind, P.fac[i].d, P.fac[i].s1, P.fac[i].s2);
  for (int i = 0; i < P.nfwd; ++i)
    printf("fwd %d %d %d %d\n", P.fwd[i].kind, P.fwd[i].d, P.fwd[i].s1, P.fwd[i].s2);
  for (int i = 0; i < P.nbwd; ++i)
    printf("bwd %d %d %d %d\n", P.bwd[i].kind, P.bwd[i].d, P.bwd[i].s1, P.bwd[i].s2);
}
int main() {
  dump<ens::Hires<double>>("hires");
  dump<ens::Pollu<double>>("pollu");
  return 0;
}
"""
CHECK, RCP, MUL, FMA, DIAG = range(5)


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("plan")
    src, exe = d / "dump.cu", d / "dump"
    src.write_text(DUMP)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res, cur = {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "model":
            cur = res[f[1]] = dict(D=int(f[2]), nnz=int(f[3]), slot=[], fac=[], fwd=[], bwd=[])
        elif f[0] == "order":
            cur["order"] = [int(x) for x in f[1:]]
        elif f[0] == "slot":
            cur["slot"].append([int(x) for x in f[1:]])
        else:
            cur[f[0]].append(tuple(int(x) for x in f[1:]))
    for p in res.values():
        p["slot"] = np.array(p["slot"])
    return res


def jac_pattern(model, D):
    P, _, _ = workloads.stiff(model, 4, seed=3)
    rng = np.random.default_rng(0)
    S = np.zeros((D, D), bool)
    for i in range(6):
        S |= oracle.jac_u(model, rng.uniform(0.1, 1.0, D), P[i % 4]) != 0
    return S


def min_degree(S):
    D = len(S)
    G = S | S.T | np.eye(D, dtype=bool)
    alive, order = list(range(D)), []
    for _ in range(D):
        v = min(alive, key=lambda x: (G[x, alive].sum(), x))
        nb = [u for u in alive if G[v, u] and u != v]
        for a in nb:
            for b in nb:
                G[a, b] = True
        order.append(v)
        alive.remove(v)
    return order


def symbolic_fill(S, order):
    D = len(S)
    F = S[np.ix_(order, order)] | np.eye(D, dtype=bool)
    for k in range(D):
        for r in range(k + 1, D):
            if F[r, k]:
                F[r, k + 1:] |= F[k, k + 1:]
    return F


@pytest.mark.parametrize("model,D", [("hires", 8), ("pollu", 20)])
def test_order_and_fill(plans, model, D):
    p = plans[model]
    assert p["D"] == D
    S = jac_pattern(model, D)
    order = min_degree(S)
    assert p["order"] == order
    F = symbolic_fill(S, order)
    np.testing.assert_array_equal(p["slot"] >= 0, F)
    assert p["nnz"] == F.sum()
    # slots numbered row-major over the filled pattern
    assert list(p["slot"][F]) == list(range(F.sum()))
    if model == "pollu":
        assert F.sum() == 109  # against 262 in natural order with partial pivoting


@pytest.mark.parametrize("model,D", [("hires", 8), ("pollu", 20)])
def test_operation_lists_factor_and_solve(plans, model, D):
    p = plans[model]
    order, slot = p["order"], p["slot"]
    P, _, _ = workloads.stiff(model, 4, seed=5)
    rng = np.random.default_rng(1)
    for trial in range(4):
        J = oracle.jac_u(model, rng.uniform(0.01, 2.0, D), P[trial])
        W = np.eye(D) - 10.0 ** rng.uniform(-3, 1) * J
        Wp = W[np.ix_(order, order)]
        a = np.zeros(p["nnz"])
        a[slot[slot >= 0]] = Wp[slot >= 0]
        checked = set()
        for kind, d, s1, s2 in p["fac"]:
            if kind == CHECK:
                checked.add((d, s1))
            elif kind == RCP:
                a[d] = 1.0 / a[d]
            elif kind == MUL:
                a[d] *= a[s1]
            else:
                assert kind == FMA
                a[d] -= a[s1] * a[s2]
        # every entry below a pivot is checked against that pivot
        for k in range(D):
            for r in range(k + 1, D):
                if slot[r, k] >= 0:
                    assert (slot[k, k], slot[r, k]) in checked
        # the factors: L unit lower, U with its diagonal stored inverted
        L, U = np.eye(D), np.zeros((D, D))
        for r in range(D):
            for c in range(D):
                if slot[r, c] < 0:
                    continue
                v = a[slot[r, c]]
                if r > c:
                    L[r, c] = v
                elif r == c:
                    U[r, c] = 1.0 / v
                else:
                    U[r, c] = v
        np.testing.assert_allclose(L @ U, Wp, rtol=1e-12, atol=1e-12 * np.abs(Wp).max())
        b = rng.normal(size=D)
        y = b[order].copy()
        for kind, d, s1, s2 in p["fwd"]:
            y[d] -= a[s1] * y[s2]
        for kind, d, s1, s2 in p["bwd"]:
            if kind == DIAG:
                y[d] *= a[s1]
            else:
                y[d] -= a[s1] * y[s2]
        x = np.empty(D)
        x[order] = y
        ref = np.linalg.solve(W, b)
        np.testing.assert_allclose(x, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
