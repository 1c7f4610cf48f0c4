"""GPU parity of ft_digest (standalone per-block CRC32C) against the oracle's
block CRC, for ragged sizes and several block sizes."""
import numpy as np
import pytest

import oracle

from _gpu import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("block", [4096, 8192, 3 * 4096, 65536])
def test_digest_sizes(block):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    rng = np.random.default_rng(block)
    for nbytes in (1, 15, 16, 17, 4095, 4096, 4097, 3 * 4096 + 1000, block - 1, block, block + 1,
                   5 * block + 123, (1 << 20) + 3):
        b = rng.integers(0, 256, size=nbytes, dtype=np.uint8)
        dev = to_dev(b)
        out = fv.digest(dev, block)
        torch.cuda.synchronize()
        ref = oracle.block_crc32c(b, block)
        assert np.array_equal(out.cpu().numpy().view(np.uint32)[:ref.size], ref), (block, nbytes)


def test_digest_matches_vote_crc():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal(1 << 20).astype(np.float32)).cuda()
    out, crc, _ = fv.vote([x, x.clone(), x.clone()], 1e-6, 1e-5)
    d = fv.digest(out)
    torch.cuda.synchronize()
    assert torch.equal(crc, d)


def test_digest_check_value():
    from paper_1405_2912_b300 import ftvote as fv
    import torch
    b = np.frombuffer(b"123456789", dtype=np.uint8)
    out = fv.digest(to_dev(b))
    torch.cuda.synchronize()
    assert int(out.cpu().numpy().view(np.uint32)[0]) == 0xE3069283
