"""The row-band split of one image across ranks (bench.py --split rows),
emulated on one GPU: each band is a view of the image with the whole image's
plane strides, convolved by its own plan reading its 2-row halos from the
source; the bands together equal the whole-image result bit for bit, which
the other tests check against the FP64 oracle."""
import numpy as np
import pytest

from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3, 5])
def test_bands_equal_whole_image(world):
    import torch

    import bench
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    P, H, W = 3, 517, 300
    A = U.to_dev(synth.image(90 + world, H, W))
    k = synth.kernel_normalised(90)
    whole = torch.empty((P, H - 4, W - 4), dtype=torch.float32, device="cuda")
    plan = sc5.Plan(P, H, W, W, W - 4)
    plan.run(A, whole, k)
    plan.close()
    bands = U.empty_dev((P, H - 4, W - 4), "f32")
    for rank in range(world):
        r0, r1 = bench.row_band(H - 4, world, rank)
        band = sc5.Plan(P, r1 - r0 + 4, W, W, W - 4, in_plane_stride=H * W, out_plane_stride=(H - 4) * (W - 4))
        band.run(A[:, r0:, :], bands[:, r0:, :], k)
        band.close()
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    assert np.array_equal(bands.cpu().numpy(), whole.cpu().numpy())
