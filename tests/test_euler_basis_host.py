"""The closed-form characteristic basis the GPU uses (csrc/euler_basis.cuh,
1-D and 2-D) evaluated on the host: L R = I, and L J R is diagonal with the
eigenvalues u.n - c, u.n, (u.n,) u.n + c for J the finite-difference Jacobian
of the oracle's normal flux -- an independent check of both closed forms."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import wlseno_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_02694_gb300", "csrc")
GAMMA = 1.4


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
    exe = str(tmp_path_factory.mktemp("basis") / "euler_basis_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-w", os.path.join(ROOT, "tests", "euler_basis_probe.cpp"),
                    "-I", CSRC, "-I", cuda_inc, "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("dim", [1, 2])
def test_closed_form_basis_diagonalises_the_jacobian(probe, dim):
    rng = np.random.default_rng(21 + dim)
    C = dim + 2
    states, normals, lines = [], [], []
    for _ in range(8):
        rho, p = rng.uniform(0.2, 2.0), rng.uniform(0.1, 2.0)
        vel = rng.uniform(-1, 1, dim)
        U = np.concatenate([[rho], rho * vel, [p / (GAMMA - 1) + 0.5 * rho * float(vel @ vel)]])
        if dim == 1:
            n = np.array([rng.choice([-1.0, 1.0])])
        else:
            a = rng.uniform(0, 2 * math.pi)
            n = np.array([math.cos(a), math.sin(a)])
        states.append(U)
        normals.append(n)
        lines.append(f"{dim} {GAMMA!r} " + " ".join(repr(float(v)) for v in [*U, *n]))
    out = subprocess.run([probe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.strip().split("\n")
    for U, n, line in zip(states, normals, out):
        vals = np.array([float(v) for v in line.split()])
        L, R = vals[:C * C].reshape(C, C), vals[C * C:].reshape(C, C)
        assert np.allclose(L @ R, np.eye(C), atol=1e-12)
        J = np.empty((C, C))
        for k in range(C):
            h = 1e-6 * max(1.0, abs(U[k]))
            e = np.zeros(C)
            e[k] = h
            J[:, k] = (O.euler_normal_flux(U + e, n, GAMMA) - O.euler_normal_flux(U - e, n, GAMMA)) / (2 * h)
        rho, vel, p = O.euler_primitive(U, GAMMA)
        un, c = float(vel @ n), math.sqrt(GAMMA * p / rho)
        lam = [un - c, un, un + c] if dim == 1 else [un - c, un, un, un + c]
        assert np.allclose(L @ J @ R, np.diag(lam), atol=1e-6)
