"""The GPU twin of the cell-body generator (used where the volume is too large
to generate on the host cores) against the CPU generator it restates: the
same cells, the same values up to FP32 rounding at sphere boundaries and in
the noise."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_gpu_cell_generator_matches_the_cpu_generator():
    import torch
    N, z0, nz = 256, 40, 24
    ref = synth.cells_u8_box(N, 0, 0, z0, N, N, nz, seed=1004, cell=64)
    out = torch.empty((nz, N, N), dtype=torch.uint8, device="cuda")
    synth.cells_u8_device(N, out.data_ptr(), seed=1004, cell=64, z0=z0, nz=nz)
    got = out.cpu().numpy()
    diff = got.astype(np.int32) - ref.astype(np.int32)
    assert np.count_nonzero(diff) <= 2e-3 * diff.size, np.count_nonzero(diff)
    # off-by-one rounding of the noisy value, or a boundary voxel between
    # interior, membrane and background
    assert np.count_nonzero(np.abs(diff) > 1) <= 5e-4 * diff.size
    # the structure is there: background, interiors and membranes
    assert (np.abs(got.astype(int) - 230) < 25).mean() > 0.01 and (got < 60).mean() > 0.2
