"""The library's cell reordering (csrc/reorder.cpp: cells sorted along the
Hilbert curve of their centroids) compiled as host C++: the order is a
permutation; on a 2^k x 2^k (and 2^k cubed) grid of points consecutive
points along it are grid neighbours, the defining property of a Hilbert
curve; and on a randomly shuffled jittered triangle mesh it brings the
stencil neighbours of the 1-ring close in index again."""
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
    exe = str(tmp_path_factory.mktemp("reorder") / "reorder_probe")
    subprocess.run([cxx, "-std=c++17", "-O2", "-w", os.path.join(ROOT, "tests", "reorder_probe.cpp"),
                    os.path.join(CSRC, "reorder.cpp"), "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", cuda_inc, "-o", exe], check=True)
    return exe


def order_of(probe, vertices, cells, period):
    dim = vertices.shape[1]
    lines = [f"{dim} {len(vertices)} {len(cells)}"]
    lines += [" ".join(repr(float(x)) for x in v) for v in vertices]
    lines += [" ".join(str(int(c)) for c in cell) for cell in cells]
    lines.append(" ".join(repr(float(p)) for p in period))
    out = subprocess.run([probe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return np.array([int(x) for x in out.stdout.split()])


def point_cells(points, eps=1e-3):
    """A tiny simplex at every point (its centroid is the point shifted by eps/(d+1))."""
    n, d = points.shape
    verts, cells = [], []
    for k, p in enumerate(points):
        verts.append(p)
        for a in range(d):
            q = p.copy()
            q[a] += eps
            verts.append(q)
        cells.append(list(range(k * (d + 1), (k + 1) * (d + 1))))
    return np.array(verts), np.array(cells)


@pytest.mark.parametrize("dim,k", [(2, 4), (2, 5), (3, 3)])
def test_consecutive_points_are_grid_neighbours(probe, dim, k):
    side = 2 ** k
    grid = np.stack(np.meshgrid(*[np.arange(side)] * dim, indexing="ij"), axis=-1).reshape(-1, dim).astype(float)
    rng = np.random.default_rng(dim * 10 + k)
    grid = grid[rng.permutation(len(grid))]
    verts, cells = point_cells(grid)
    order = order_of(probe, verts, cells, np.zeros(dim))
    assert sorted(order.tolist()) == list(range(len(grid)))
    path = grid[order]
    steps = np.abs(np.diff(path, axis=0)).sum(axis=1)
    assert np.all(steps == 1.0), np.unique(steps)


def test_shuffled_mesh_regains_locality(probe):
    mesh = synth.tri_mesh(32, jitter=0.2, seed=1)
    rng = np.random.default_rng(7)
    shuffle = rng.permutation(mesh.n_cells)
    cells = mesh.cells[shuffle]
    order = order_of(probe, mesh.vertices, cells, mesh.period)
    assert sorted(order.tolist()) == list(range(mesh.n_cells))
    new_of_old = np.empty_like(order)
    new_of_old[order] = np.arange(len(order))
    stencils, _ = O.build_stencils(cells, 1.0, 2)

    def spread(rank):
        return float(np.median([abs(rank[i] - rank[j]) for i in range(len(cells)) for j in stencils[i][1:]]))

    shuffled = spread(np.arange(len(cells)))
    reordered = spread(new_of_old)
    original = spread(np.argsort(shuffle))  # the generator's row order
    assert reordered < shuffled / 20
    assert reordered <= 2 * original
