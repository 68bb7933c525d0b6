"""The library's square-root-free Givens fold (csrc/k_recon_tpc.cuh, the
thread-per-cell least-squares solver, FP64) compiled as host C++ and
checked against library least squares: random weighted problems of the
bench's shape (37 x 10) and of a square one give numpy's solution, and the
conditioning estimate sqrt(qmax/qmin) is at most the condition number of
the column-scaled weighted matrix W A S (Sec. 3.3.2), the bound the flag
threshold relies on; the second estimate (the LINPACK-style inverse
estimate of the column-scaled factor) is at most ||(W A S)^-1||_1 and
routes to the pivoted path every cell whose rank the rule of Sec. 3.3.2
truncates, also on weighted stencils where the spread stays moderate."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_02694_gb300", "csrc")
M = 10


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = None
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(cand, "include")
            break
    if cxx is None or cuda_inc is None:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("fold") / "fold_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-w", "-ffp-contract=off", os.path.join(ROOT, "tests", "fold_probe.cpp"),
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", cuda_inc, "-o", exe], check=True)
    return exe


def solve(probe, problems, args=()):
    lines = []
    for w, A, b in problems:
        lines.append(str(len(w)))
        for t in range(len(w)):
            lines.append(" ".join(repr(float(v)) for v in [w[t], *A[t], b[t]]))
    out = subprocess.run([probe, *args], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    res = []
    for k in range(len(problems)):
        x = np.array([float(v) for v in out[3 * k].split()[1:]])
        qmax, qmin = (float(v) for v in out[3 * k + 1].split()[1:])
        est = float(out[3 * k + 2].split()[1])
        res.append((x, qmax, qmin, est))
    return res


def test_fold_solves_weighted_least_squares(probe):
    rng = np.random.default_rng(3)
    problems = []
    for n in (37, 37, 37, 10, 19):
        A = rng.normal(size=(n, M)) * np.exp(rng.uniform(-2, 2, M))[None, :]  # uneven column scales
        w = np.exp(rng.uniform(-4, 0, n))                                     # weights over 4 decades
        b = rng.normal(size=n)
        problems.append((w, A, b))
    for (w, A, b), (x, qmax, qmin, est) in zip(problems, solve(probe, problems)):
        WA = w[:, None] * A
        want = np.linalg.lstsq(WA, w * b, rcond=None)[0]
        S = 1.0 / np.linalg.norm(WA, axis=0)
        kappa = np.linalg.cond(WA * S[None, :])
        assert np.max(np.abs(x - want)) <= 1e-9 * kappa * max(1.0, np.max(np.abs(want)))
        assert np.sqrt(qmax / qmin) <= kappa * (1 + 1e-9)
        # est = ||z||_inf for R_B^T z = e, |e_k| = 1: at most ||R_B^-T||_inf = ||R_B^-1||_1
        inv1 = np.max(np.sum(np.abs(np.linalg.inv(np.linalg.qr(WA * S[None, :], mode="r"))), axis=0))
        assert 1.0 <= est <= inv1 * (1 + 1e-5), (est, inv1)


def test_zero_weight_rows_leave_the_solution_unchanged(probe):
    rng = np.random.default_rng(4)
    A = rng.normal(size=(20, M))
    b = rng.normal(size=20)
    w = np.ones(20)
    w0 = w.copy()
    w0[5:9] = 0.0
    (x_all, _, _, _), (x_zero, _, _, _) = solve(probe, [(w, A, b), (w0, A, b)])
    keep = np.ones(20, dtype=bool)
    keep[5:9] = False
    want = np.linalg.lstsq(A[keep], b[keep], rcond=None)[0]
    assert np.max(np.abs(x_zero - want)) <= 1e-10 * max(1.0, np.max(np.abs(want)))
    assert not np.allclose(x_all, x_zero)


def test_rank_deficient_system_is_flagged(probe):
    """Two equal columns: the conditioning estimate blows up (the cell would
    go to the pivoted path), while a well-conditioned copy stays small."""
    rng = np.random.default_rng(5)
    A = rng.normal(size=(37, M))
    B = A.copy()
    B[:, 7] = B[:, 3]
    w = np.ones(37)
    b = rng.normal(size=37)
    (_, q1, q0, e1), (_, p1, p0, e2) = solve(probe, [(w, A, b), (w, B, b)])
    assert math.sqrt(q1 / q0) < 1e2 and e1 < 1e2
    assert not (p1 <= 1e12 * p0)  # beyond any flag threshold (1e6 squared)
    assert not (e2 <= 1e6)


def test_truncated_cells_reach_the_pivoted_path(probe):
    """Weighted stencils dominated by cells with collinear centroids (the
    unjittered grid, averages of sin(2 pi (x + y)) equal along x + y = const,
    eps = 1e-12, weights spanning 1e13 to 1e15): the oracle's rank rule
    (rank_tol 1e-10) truncates every cell, and every cell reaches the
    pivoted path of the FP64 kernel: its spread or inverse estimate exceeds
    the pivot bound (1e6), or its weights span more than 1e6 (the bound of
    the fold's rounding, which leaves some of these cells with a moderate
    diagonal where the true factor nearly vanishes)."""
    from oracle import wlseno_oracle as O
    from paper_1602_02694_gb300 import synth
    mesh = synth.tri_mesh(12, jitter=0.0, seed=1)
    ubar = synth.cell_averages(mesh, lambda P: np.sin(2 * np.pi * (P[:, 0] + P[:, 1])), k=6)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.BURGERS, eps=1e-12)
    problems, ranks = [], []
    for i in range(prob.N):
        S = prob.stencils[i]
        face = set(prob.face_nbrs[i])
        uS = np.array([ubar[j] for j in S])
        omega = O.wls_eno_weights(uS, [j in face for j in S], prob.geo.h[i], prob.eps, prob.alpha_c)
        problems.append((omega, prob.A(i), uS - uS[0]))
        ranks.append(prob.reconstruct_cell(ubar, i)[1])
    ranks = np.array(ranks)
    assert np.all(ranks < M)
    res = solve(probe, problems)
    spread_w = [np.max(w) / np.min(w) for w, _, _ in problems]
    routed = [not (qmax <= 1e12 * qmin) or not (est <= 1e6) or not (sw <= 1e6)
              for (_, qmax, qmin, est), sw in zip(res, spread_w)]
    assert all(routed)
    # the weight spread is what catches the cells both estimates miss
    assert any(qmax <= 1e12 * qmin and est <= 1e6 for _, qmax, qmin, est in res)


def test_first_row_folded_into_row_zero_only(probe):
    # the centre row folded into a fresh factor as far as its row 0 (the
    # constant column is 1 in every moment row): the same least-squares
    # solution as the full fold, and the same conditioning tests, for
    # weights over four decades, the centre weight among them
    rng = np.random.default_rng(8)
    problems = []
    for n in (13, 13, 37, 19):
        A = rng.normal(size=(n, M)) * np.exp(rng.uniform(-2, 2, M))[None, :]
        A[:, 0] = 1.0
        A[0, 1:3] = 0.0  # the centre row's first moments about its own centroid
        w = np.exp(rng.uniform(-4, 0, n))
        b = rng.normal(size=n)
        b[0] = 0.0
        problems.append((w, A, b))
    full = solve(probe, problems)
    head = solve(probe, problems, ("first",))
    for (w, A, b), (x0, qmax0, qmin0, est0), (x1, qmax1, qmin1, est1) in zip(problems, full, head):
        WA = w[:, None] * A
        want = np.linalg.lstsq(WA, w * b, rcond=None)[0]
        S = 1.0 / np.linalg.norm(WA, axis=0)
        kappa = np.linalg.cond(WA * S[None, :])
        scale = max(1.0, np.max(np.abs(want)))
        assert np.max(np.abs(x1 - want)) <= 1e-9 * kappa * scale
        assert np.max(np.abs(x1 - x0)) <= 1e-9 * kappa * scale
        assert abs(qmax1 / qmin1 - qmax0 / qmin0) <= 1e-9 * qmax0 / qmin0
        assert abs(est1 - est0) <= 1e-5 * est0
