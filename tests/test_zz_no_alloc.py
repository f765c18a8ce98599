"""md_bin_cells_noalloc: the cell binner for callers that cannot allocate
device memory (a fixed memory pool or budget that may not grow).  Its output
must equal the oracle's cell bins (wrap, cell formula, stable counting sort)
and what md_cells reports after md_create for the same positions, on
consecutive calls that share the library's one static scratch array.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

import oracle as O
from paper_2405_07898_gb300 import binding, inputs as I

pytestmark = pytest.mark.gpu


def _bins_via_context(system):
    with binding.MD(system, precision="fp64") as md:
        return md.cells()


def _bins_noalloc(system, stream):
    import torch
    nc = np.floor(system.box / system.pot.r_list).astype(np.int64)
    ncells = int(np.prod(nc))
    pos = torch.from_numpy(np.ascontiguousarray(system.pos)).to("cuda")
    start = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
    atoms = torch.full((max(system.n, 1),), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = binding.bin_cells_noalloc(system.box, system.pot.r_list, system.n, pos.data_ptr(),
                                   start.data_ptr(), atoms.data_ptr(), stream.cuda_stream)
    assert rc == 0
    stream.synchronize()
    return start.cpu().numpy(), atoms.cpu().numpy()[: system.n]


def _bins_oracle(system):
    w = O.wrap(system.pos, system.box)
    _, start, atoms = O.cells(w, system.box, system.pot.r_list)
    return start, atoms


def test_no_alloc_binner_matches_oracle_and_md_cells_on_consecutive_calls():
    import torch
    stream = torch.cuda.Stream()
    a = I.bcc_2000_fp64()
    b = I.thermal_system(I.BCC_TA_LIKE, (12, 11, 13), 0.05, 500.0, 4242)
    # wrapped-out-of-box input positions exercise the wrap
    b.pos[::7] += b.box * np.array([1.0, -1.0, 2.0])
    for system in (a, b, a):  # consecutive calls share (and must clear) the scratch array
        start_o, atoms_o = _bins_oracle(system)
        start, atoms = _bins_noalloc(system, stream)
        np.testing.assert_array_equal(start, start_o)
        np.testing.assert_array_equal(atoms, atoms_o)
        _, start_ref, atoms_ref = _bins_via_context(system)
        np.testing.assert_array_equal(start, start_ref)
        np.testing.assert_array_equal(atoms, atoms_ref)


def test_no_alloc_binner_crowded_cell_and_largest_size():
    """Every atom in a handful of cells (the order inside a cell is a sort,
    not a per-cell walk), and the largest accepted atom count, against the
    oracle."""
    import torch
    stream = torch.cuda.Stream()
    rng = np.random.Generator(np.random.PCG64(2405))
    box = np.array([20.0, 21.0, 22.0])
    crowd = rng.random((50000, 3)) * np.array([0.5, 0.5, 0.5]) + np.array([1.0, 10.0, 20.0])
    pot = I.johnson_potential(I.BCC_TA_LIKE, n_knots=50)
    s1 = I.System(box=box, pos=crowd, vel=np.zeros_like(crowd), types=np.zeros(len(crowd), np.int32), pot=pot)
    big = rng.random((1 << 18, 3)) * np.array([100.0, 90.0, 80.0])
    s2 = I.System(box=np.array([100.0, 90.0, 80.0]), pos=big, vel=np.zeros_like(big),
                  types=np.zeros(len(big), np.int32), pot=pot)
    for system in (s1, s2):
        start_o, atoms_o = _bins_oracle(system)
        start, atoms = _bins_noalloc(system, stream)
        np.testing.assert_array_equal(start, start_o)
        np.testing.assert_array_equal(atoms, atoms_o)


def test_no_alloc_binner_rejects_sizes_beyond_its_maximum():
    box = np.array([400.0, 400.0, 400.0])  # 83^3 cells > 65,536
    assert binding.bin_cells_noalloc(box, 4.8, 10, 0, 0, 0, 0) == -8  # MD_ERR_CAPACITY
    box = np.array([100.0, 100.0, 100.0])
    assert binding.bin_cells_noalloc(box, 4.8, 300000, 0, 0, 0, 0) == -8
