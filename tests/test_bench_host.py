"""Host-side pieces of bench.py on the CPU: the oracle baseline's patch
sub-meshes reproduce the whole mesh's oracle results for the patch cells
bit for bit, and the algorithmic byte and flop counts follow their
formulas for the bench workload."""
import os
import sys

import numpy as np

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_patch_submesh_reproduces_the_whole_mesh_bitwise():
    n, patch, pad = 24, 6, 6
    mesh = synth.tri_mesh(n, jitter=0.2, seed=1)
    u = synth.burgers_2d_initial(mesh)
    i0 = j0 = 9
    sub, local, glob = bench.patch_submesh(mesh, i0, j0, patch=patch, pad=pad)
    whole = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.BURGERS)
    part = O.Problem(sub.vertices, sub.cells, sub.period, p=4, ring=2.0, pde=O.BURGERS)
    us = u[glob]
    for c in local:
        g = int(glob[c])
        assert [int(glob[k]) for k in part.stencils[c]] == list(whole.stencils[g])
        a = part.reconstruct_cell(us, c)[0]
        b = whole.reconstruct_cell(u, g)[0]
        assert np.array_equal(a, b), c
        for f in range(3):
            ca, fa = part.sib[c, f]
            cb, fb = whole.sib[g, f]
            assert int(glob[ca]) == cb and fa == fb


def test_algorithmic_counts_of_the_bench_workload():
    n, m, npts, dim = 37, 10, 6, 2
    stored = bench.algorithmic_bytes_per_cell(n, m, npts, dim, 4)
    fly = bench.algorithmic_bytes_per_cell(n, m, npts, dim, 4, on_the_fly=True)
    tail = 4 * n + 8 + 8 + 4 * (dim + 1) + npts * dim * 4 + 8 * npts
    assert stored == n * m * 4 + tail
    assert fly == n * dim * 4 + (m - 1 - dim) * 4 + tail
    assert fly < stored / 2.5
    assert 13_000 < bench.algorithmic_flops_per_cell(n, m, npts) < 16_000


def test_patch_sweep_is_one_stage_however_it_is_split():
    """The baseline's patch sweep: one sweep updates every patch cell by
    dt times the oracle's residual of the sub-mesh, and splitting sweeps into
    steps of any size changes nothing."""
    n, patch, pad = 24, 6, 6
    mesh = synth.tri_mesh(n, jitter=0.2, seed=1)
    u0 = synth.burgers_2d_initial(mesh)
    a = bench._PatchSweep(mesh, u0, 9, 9, patch=patch, pad=pad)
    b = bench._PatchSweep(mesh, u0, 9, 9, patch=patch, pad=pad)
    cells = a.cells
    start = a.u.copy()
    a.advance(len(cells))
    for k in (5, 30, len(cells) - 35):
        b.advance(k)
    assert np.array_equal(a.u, b.u)
    L = O.residual(a.prob, start)
    want = start[cells] + a.dt * L[cells]
    assert np.max(np.abs(a.u[cells] - want)) <= 1e-15 * np.max(np.abs(start))
    a.advance(len(cells) + 17)
    for k in (1, len(cells) + 16):
        b.advance(k)
    assert np.array_equal(a.u, b.u) and a.cursor == b.cursor == 17


def test_reference_arm_runs_the_requested_steps(monkeypatch):
    monkeypatch.setattr(bench, "PATCH", 4)
    monkeypatch.setattr(bench, "PATCH_PAD", 6)
    mesh = synth.tri_mesh(24, jitter=0.2, seed=1)
    u0 = synth.burgers_2d_initial(mesh)
    done, elapsed, k = bench._oracle_patch_worker((mesh, u0, 9, 9, 0.2, 2, 3))
    assert k >= 1 and done == 3 * k and elapsed > 0.0


def test_cpu_baseline_times_whole_stages(monkeypatch):
    monkeypatch.setattr(bench, "PATCH", 4)
    monkeypatch.setattr(bench, "PATCH_PAD", 6)
    mesh = synth.tri_mesh(24, jitter=0.2, seed=1)
    u0 = synth.burgers_2d_initial(mesh)
    done, elapsed, k = bench._oracle_patch_worker((mesh, u0, 9, 9, 0.05, 0, None))
    assert k == 2 * 4 * 4 and done % k == 0 and done >= k and elapsed >= 0.05


def test_euler_reference_arm_times_whole_oracle_steps():
    """The Euler workload's oracle baseline: K timed whole RK3 steps of a
    transmissive sub-mesh of the grid (3 cell-stages per cell and step),
    and the sub-mesh's oracle step equals the oracle's step of that mesh."""
    done, elapsed, cells = bench._oracle_euler_worker((48, 3, 24, 24, 0.3, 1, 2))
    assert cells >= 8 and done == 3 * cells * 2 and elapsed > 0.0
    done, elapsed, cells = bench._oracle_euler_worker((48, 3, 24, 24, 0.05, 0, None))
    assert done % (3 * cells) == 0 and done >= 3 * cells and elapsed >= 0.05


def test_euler_and_flux_algorithmic_bytes():
    # 2-D Euler, p = 3 on the 1-ring: 13 offset records, one own-moment record
    n, m, npts, dim = 13, 6, 6, 2
    fly = bench.euler_recon_bytes_per_cell(n, m, npts, dim, True)
    assert fly == 13 * 16 + 16 + 4 + 8 * 4 + 8 + 12 + 6 * 2 * 4 + 1 + 4 * 4 * 6
    stored = bench.euler_recon_bytes_per_cell(n, m, npts, dim, False)
    assert stored == 13 * 32 + 4 + 32 + 8 + 12 + 48 + 1 + 96
    # scalar double-float flux: deviations, pairs of u and u0, neighbours,
    # facet records, 1/|tau|, FP64 state and pairs written
    assert bench.flux_bytes_per_cell(2, 6, 1, False) == 6 * 4 + 8 + 8 + 12 + 48 + 8 + 16
    # FP32 Euler: the traces of the four components instead of deviations
    # and positivity flags
    assert bench.flux_bytes_per_cell(2, 6, 4, True) == 4 * (24 + 16) + 12 + 48 + 8 + 4 * 16


def test_measured_traffic_only_for_the_captured_kernel_sources(monkeypatch):
    # the stored per-cell DRAM bytes scale with the workload's cells while
    # the sources match the capture's digest, and vanish once they do not
    key = ("euler1024", "fp32_bulk", "reconstruct", False)
    per_cell = bench.TRAFFIC_BYTES_PER_CELL[key][0]
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_DIGEST", bench.kernel_sources_digest())
    assert bench.traffic_per_launch(*key, 2097152) == per_cell * 2097152
    assert bench.traffic_per_launch("batched48", "fp32_bulk", "reconstruct", True, 10) is None
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_DIGEST", "0" * 12)
    assert bench.traffic_per_launch(*key, 2097152) is None
    # every capture is within a few times the algorithmic bytes of its kernel
    # (more would mean the capture did not run the kernel the key names)
    alg = bench.euler_recon_bytes_per_cell(13, 6, 6, 2, False)
    assert 0.8 * alg < per_cell < 1.5 * alg


def test_source_digest_ignores_comments_not_code():
    # comments and white-space runs leave the stripped source unchanged;
    # code, and comment markers inside string literals, do not
    a = 'int f(int x) {  // twice\n  return 2 * x; /* doubled */ }\nconst char* s = "a // b";'
    b = "int f(int x) { return 2 * x; }\n// another comment\nconst char* s = \"a // b\";"
    assert bench.strip_c_comments(a) == bench.strip_c_comments(b)
    assert bench.strip_c_comments(a) != bench.strip_c_comments(a.replace("2 * x", "3 * x"))
    assert "a // b" in bench.strip_c_comments(a)
