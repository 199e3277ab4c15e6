"""The CUDA path's Philox4x32-10 against the oracle's independent
implementation (itself pinned to the Random123 known-answer vectors):
bit-exact on 10^6 counters, both device forms (the step's precomputed round
keys, the resets' inline key schedule), keys including the extremes."""
import numpy as np
import pytest
import torch

from gpu_helpers import DEV
from oracle import oracle as O
from paper_2306_09537_gb300 import qs

pytestmark = pytest.mark.gpu


def test_philox_bit_exact_against_oracle():
    rng = np.random.default_rng(2306)
    n = 1_000_000
    ctr = rng.integers(0, 2 ** 32, size=(n, 3), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0], [0xFFFFFFFF] * 3, [1, 2, 3], [0xFFFFFFFF, 0, 0xFFFFFFFF]]
    # counters of the step's own layout: (tick, drone or env, tag << 16 | sub << 8 | block)
    ctr[4:1004, 0] = np.arange(1000)
    ctr[4:1004, 2] = (3 << 16) | (1 << 8)
    ctr4 = np.concatenate([ctr, np.zeros((n, 1), np.uint32)], axis=1)
    ctr_dev = torch.from_numpy(ctr.view(np.int32)).to(DEV)
    out = torch.empty(n, 4, dtype=torch.int32, device=DEV)
    keys = [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (1, 0)] + [tuple(int(x) for x in rng.integers(0, 2 ** 32, 2)) for _ in range(3)]
    for key0, key1 in keys:
        want = O.philox4x32_10_batch(ctr4, [key0, key1])
        for variant in (0, 1):
            qs.qs_philox4x32_10(ctr_dev, key0, key1, out, variant)
            torch.cuda.synchronize()
            got = out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want), (key0, key1, variant, int((got != want).any(axis=1).sum()))


def test_philox_rejects_bad_arguments():
    ctr = torch.zeros(4, 3, dtype=torch.int32, device=DEV)
    out = torch.zeros(4, 4, dtype=torch.int32, device=DEV)
    with pytest.raises(qs.QSError):
        qs.qs_philox4x32_10(ctr, 1, 2, out, variant=2)
    with pytest.raises(qs.QSError):
        qs.qs_philox4x32_10(ctr, 1, 2, None)  # no output buffer
