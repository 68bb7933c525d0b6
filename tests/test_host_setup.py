"""The library's native host setup (csrc/host_mesh.cpp) on the CPU, built
with the host compiler into a small probe (tests/host_setup_probe.cpp) and
compared with the oracle: k-ring stencils bit-exact (periodic and
transmissive, 1-D to 3-D, radius cut, short-stencil growth), geometry to
rounding, facet neighbours, and the balanced-stencil candidate rings; plus
the documented errors for an inverted cell, a facet shared by three cells,
a vertex index out of range, a repeated vertex and a stencil smaller than
m."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_02694_gb300", "csrc")


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
    exe = str(tmp_path_factory.mktemp("probe") / "host_setup_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", os.path.join(ROOT, "tests", "host_setup_probe.cpp"),
                    os.path.join(CSRC, "host_mesh.cpp"), "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", cuda_inc, "-o", exe], check=True)
    return exe


def run(probe, mesh, p, ring, radius_cut=0.0, min_rows=0, balance_steps=0):
    d = mesh.vertices.shape[1]
    head = f"{d} {mesh.vertices.shape[0]} {mesh.cells.shape[0]} {p} {ring!r} {radius_cut!r} {min_rows} {balance_steps}"
    body = " ".join(repr(float(x)) for x in np.asarray(mesh.period, dtype=np.float64).ravel())
    body += "\n" + " ".join(repr(float(x)) for x in mesh.vertices.ravel())
    body += "\n" + " ".join(str(int(x)) for x in mesh.cells.ravel())
    out = subprocess.run([probe], input=head + "\n" + body + "\n", capture_output=True, text=True, check=True).stdout
    lines = out.strip().split("\n")
    status = int(lines[0].split()[1])
    res = {"status": status, "message": lines[0].split(" ", 2)[2]}
    for line in lines[1:]:
        parts = line.split()
        vals = parts[2:]
        res[parts[0]] = np.array([float(v) if ("." in v or "e" in v or "n" in v) else int(v) for v in vals])
    return res


CASES = [
    ("tri8_p4_ring2", lambda: synth.tri_mesh(8, seed=4), 4, 2.0, 0.0, 15),
    ("tri7_p3_open", lambda: synth.tri_mesh(7, periodic=False, seed=12), 3, 1.0, 0.0, 9),
    ("tri6_p3_half", lambda: synth.tri_mesh(6, seed=5), 3, 1.5, 0.0, 9),
    ("tet3_p3", lambda: synth.tet_mesh(3, seed=15), 3, 2.0 / 3.0, 0.0, 15),
    ("tet3_p3_cut", lambda: synth.tet_mesh(3, seed=16), 3, 2.0 / 3.0, 0.95, 15),
    ("tet3_p3_open", lambda: synth.tet_mesh(3, periodic=False, seed=14), 3, 2.0 / 3.0, 0.0, 15),
    ("line20_p5", lambda: synth.periodic_line_mesh(20, jitter=0.2, seed=6), 5, 2.0, 0.0, 5),
]


@pytest.mark.parametrize("name,make,p,ring,cut,min_rows", CASES, ids=[c[0] for c in CASES])
def test_host_setup_matches_the_oracle(probe, name, make, p, ring, cut, min_rows):
    mesh = make()
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, radius_cut=cut, min_rows=min_rows)
    steps = int(math.ceil(ring - 1e-9)) + 1
    r = run(probe, mesh, p, ring, cut, min_rows, balance_steps=steps)
    assert r["status"] == 0, r["message"]
    N, d = prob.N, prob.dim
    ptr, cols = r["row_ptr"], r["cols"]
    assert [list(cols[ptr[i]:ptr[i + 1]]) for i in range(N)] == [list(s) for s in prob.stencils]
    assert np.allclose(r["centroid"].reshape(N, d), prob.geo.centroid, rtol=0, atol=1e-15)
    assert np.allclose(r["volume"], prob.geo.volume, rtol=1e-13, atol=0)
    assert np.allclose(r["h"], prob.geo.h, rtol=1e-14, atol=0)
    assert np.allclose(r["inradius"], prob.geo.inradius, rtol=1e-13, atol=0)
    nbr = r["nbr"].reshape(N, d + 1)
    for i in range(N):
        for f in range(d + 1):
            j, fj = prob.sib[i, f]
            if j < 0:
                assert nbr[i, f] == -1
            else:
                assert (nbr[i, f] >> 2, nbr[i, f] & 3) == (j, fj), (i, f)
    bp, bi = r["bal_ptr"], r["bal_idx"]
    for i in range(0, N, max(1, N // 40)):
        want = sorted(O.k_ring(i, ["vertex"] * steps, prob.nbr) - {i})
        assert list(bi[bp[i]:bp[i + 1]]) == want, i


def test_host_setup_reports_mesh_and_stencil_errors(probe):
    mesh = synth.tri_mesh(5, seed=1)
    bad = synth.Mesh(mesh.vertices, mesh.cells[:, [0, 2, 1]].copy(), mesh.period, mesh.cell_coords, n=mesh.n)
    r = run(probe, bad, 3, 1.0)
    assert r["status"] == -2, r  # WLSENO_ERR_MESH: inverted cells
    line = synth.line_mesh(np.linspace(0.0, 1.0, 6))
    r = run(probe, line, 5, 1.0, min_rows=3)
    assert r["status"] == -3, r  # WLSENO_ERR_STENCIL: 3-cell stencils for m = 5


def test_host_setup_reports_malformed_meshes(probe):
    """The documented MESH errors: a facet shared by three cells (not a
    manifold), a vertex index out of range and a cell that repeats a vertex
    (degenerate), each reported with a message naming the problem."""
    mesh = synth.tri_mesh(4, periodic=False, seed=1)
    V, Cl = mesh.vertices, mesh.cells
    # a third triangle on the first cell's edge (v0, v1), apex beyond it
    v0, v1, v2 = (int(x) for x in Cl[0])
    apex = V[v0] + V[v1] - V[v2]
    V3 = np.vstack([V, apex, apex + 0.01])
    extra = np.array([[v1, v0, len(V)], [v1, v0, len(V) + 1]])
    cells3 = np.vstack([Cl, extra])
    # keep every cell positively oriented
    for c in range(len(Cl), len(cells3)):
        a, b, e = V3[cells3[c]]
        if (b[0] - a[0]) * (e[1] - a[1]) - (b[1] - a[1]) * (e[0] - a[0]) < 0:
            cells3[c, [0, 1]] = cells3[c, [1, 0]]
    r = run(probe, synth.Mesh(V3, cells3, mesh.period, V3[cells3], n=mesh.n), 3, 1.0, min_rows=9)
    assert r["status"] == -2 and "more than two" in r["message"], r
    bad = Cl.copy()
    bad[3, 2] = len(V) + 7
    r = run(probe, synth.Mesh(V, bad, mesh.period, mesh.cell_coords, n=mesh.n), 3, 1.0, min_rows=9)
    assert r["status"] == -2 and "out of range" in r["message"], r
    rep = Cl.copy()
    rep[5, 2] = rep[5, 1]
    r = run(probe, synth.Mesh(V, rep, mesh.period, mesh.cell_coords, n=mesh.n), 3, 1.0, min_rows=9)
    assert r["status"] == -2, r
