"""The arithmetic behind bench.py's roofline line, pinned on CPU: the algorithmic flop counts per
cell, the cell shapes they are fed, and the irreducible points of the periodic k-grid.

The counts are definitions, so the pins are hand counts of small cases and closed forms:
- a water (6 orbitals, 4 occupied, 3 atom pairs) costs 2n^3 + 9n^3 + 2n^2 n_occ + 2n^2 = 2736 flops
  per SCC iteration plus 1000 per pair;
- a Gamma-centred k x k x k grid has (k^3 + m) / 2 irreducible points under k <-> -k, where m is
  the number of points equal to their own negative (1 for odd k, 8 for even k)."""
import numpy as np
import pytest

import bench
import cavmd_synth as cs


def test_water_flops_per_iteration_and_pairs():
    assert bench._dftb_flops_per_cell(0) == pytest.approx(3000.0)
    assert bench._dftb_flops_per_cell(1) == pytest.approx(2736.0 + 3000.0)
    # linear in the iteration count, one water per entry
    it = np.array([1, 6, 7])
    np.testing.assert_allclose(bench._dftb_flops_per_cell(it), 2736.0 * it + 3000.0)


def test_cluster_flops_follow_the_water_model():
    # (H2O)_2: n = 12, n_occ = 8, 15 atom pairs
    n, no, npair = 12, 8, 15
    per_iter = 11 * n ** 3 + 2 * n * n * no + 2 * n * n
    assert bench._dftb_flops_per_cell(2, n, no, npair) == pytest.approx(2 * per_iter + 15000.0)


def test_cell_shapes_of_water_and_cluster_systems():
    w = cs.make_workload("c1")
    n, no, npair = bench._cell_shapes(w["system"])
    assert np.all(n == 6) and np.all(no == 4) and np.all(npair == 3)
    w3 = cs.make_workload("c3", n_cells=50)
    nat = np.diff(w3["system"].cell_offset)
    n, no, npair = bench._cell_shapes(w3["system"])
    np.testing.assert_array_equal(n, 2 * nat)
    np.testing.assert_array_equal(no, 4 * nat // 3)
    np.testing.assert_array_equal(npair, nat * (nat - 1) // 2)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_irreducible_kgrid_points(k):
    self_inverse = 1 if k % 2 else 8
    assert bench._kgrid_points(k) == (k ** 3 + self_inverse) // 2
    assert bench._kgrid_points(3) == 14


def test_periodic_flops_grow_with_iterations_and_cubically_with_size():
    a = bench._periodic_flops_per_cell(10, 198, 132)
    b = bench._periodic_flops_per_cell(11, 198, 132)
    c = bench._periodic_flops_per_cell(12, 198, 132)
    assert b > a and c - b == pytest.approx(b - a)   # affine in the iteration count past the first
    # every term is at most cubic in the size: doubling n (and n_occ) multiplies by at most 8
    assert bench._periodic_flops_per_cell(10, 396, 264) <= 8.0 * a * (1 + 1e-12)
    assert bench._periodic_flops_per_cell(10, 396, 264) > 4.0 * a
