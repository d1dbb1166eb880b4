"""The GPU form of the seeded input recipe (mbc_inputs/gen.cu) against the host recipe:
same counters and streams, so every entry agrees to the last few bits (the logarithm,
square root and sine/cosine are the GPU's), plain and noisy fields (needs a GPU)."""
import numpy as np
import pytest

import mbc_inputs as mi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,set_index,flavour,kappa,noise", [(3, 0, 0, 0.5, None), (100, 37, 1, 0.5, None),
                                                                 (5, 6, 1, 0.3, 1e-3)])
def test_gpu_fields_match_host_recipe(seed, set_index, flavour, kappa, noise):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V3, ts = 27, [0, 5, 47]
    ref = np.stack([mi.site_matrices(seed, set_index, flavour, t, np.arange(V3), kappa, noise) for t in ts])
    out = torch.empty(len(ts), V3, 12, 12, dtype=torch.complex128, device="cuda")
    mi.fill_device(out.data_ptr(), seed, set_index, flavour, V3, ts, kappa, noise,
                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    err = np.max(np.abs(got - ref) / np.max(np.abs(ref), axis=(1, 2, 3), keepdims=True))
    assert err <= 1e-14, err
