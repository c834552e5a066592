"""The bandwidth yardstick lb_stream_bound (the step's streaming loads and stores without its
arithmetic) copies exactly what its definition says: f_out[l](x) = f_in[l](x - c_l), periodic in
x and y, z clamped to the cell; bit-exact in both element sizes and both launch shapes."""
import numpy as np
import pytest
import torch

from oracle.lbm import C
from paper_1111_0905_gb300 import lb

pytestmark = pytest.mark.gpu


def _pulled(a):
    """a: [19, nz, ny, nx] numpy; the pull of each direction with the z clamp."""
    nz = a.shape[1]
    out = np.empty_like(a)
    for l, (cx, cy, cz) in enumerate(C):
        zs = np.clip(np.arange(nz) - cz, 0, nz - 1)
        out[l] = np.roll(np.roll(a[l], cx, axis=2), cy, axis=1)[zs]
    return out


@pytest.mark.parametrize("dtype", [torch.float32, torch.int16])
@pytest.mark.parametrize("ctas", [0, 1, 2])
def test_stream_bound_is_the_pull_copy(lblib, dtype, ctas):
    # 97,200 nodes: more than one resident wave of 2 x 152 CTAs of 256 threads (the strided loop
    # runs twice), not a multiple of 256 or of a warp row (ragged tail)
    shape = (9, 40, 270)
    n = 19 * shape[0] * shape[1] * shape[2]
    gen = torch.Generator().manual_seed(11)
    if dtype == torch.float32:
        fi, gi = (torch.rand(n, generator=gen, dtype=torch.float32) for _ in range(2))
    else:
        fi, gi = (torch.randint(-32768, 32767, (n,), generator=gen, dtype=torch.int16) for _ in range(2))
    fi_d, gi_d = fi.cuda(), gi.cuda()
    fo_d, go_d = torch.zeros_like(fi_d), torch.zeros_like(gi_d)
    occ = lb.stream_bound(fi_d, gi_d, fo_d, go_d, shape, ctas)
    torch.cuda.synchronize()
    assert occ >= 2
    for got, src in ((fo_d, fi), (go_d, gi)):
        want = _pulled(src.numpy().reshape(19, *shape))
        assert np.array_equal(got.cpu().numpy().reshape(19, *shape), want)


def test_stream_bound_refuses_more_ctas_than_fit(lblib):
    shape = (2, 2, 2)
    t = [torch.zeros(19 * 8, dtype=torch.float32, device="cuda") for _ in range(4)]
    occ = lb.stream_bound(*t, shape, 0)
    with pytest.raises(lb.LBError) as e:
        lb.stream_bound(*t, shape, occ + 1)
    assert e.value.code == -1
