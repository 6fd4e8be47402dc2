"""pnop_energy_noalloc against the context's pnop_energy.

pnop_energy_noalloc is for callers that cannot call cudaMalloc where they
need the energy: code that runs after all device memory has been handed to
another allocator or a fixed pool (a further cudaMalloc would fail), or loops
that must avoid cudaMalloc/cudaFree because they can synchronise the device.
It needs no context and keeps its reduction scratch in a fixed device array
inside the library, shared by every call.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-13  # the energy tolerance of the parity tests


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    return _lib


def _case(L, nr, M, K, Lz, seed):
    import torch
    ctx = L.Context(nr, 2 * (M + 1), 2 * (K + 1), Lz, 2000.0, 0.01, 8.0, 1.0, 0.0, 0, 1)
    r = np.array(ctx.pnop_grid_points())
    u = torch.from_numpy(synth.random_field(r, M, K, Lz, seed=seed)).to("cuda")
    W = torch.from_numpy(po.radial_weights(r)).to("cuda")
    return ctx, u, W


def test_noalloc_energy_matches_context_energy_on_two_calls(L):
    # first call on a larger field (more partial sums), second on a smaller one:
    # the second must not see what the first left in the shared scratch
    ctx1, u1, W1 = _case(L, 32, 15, 47, 50.0, seed=3)
    ctx2, u2, W2 = _case(L, 12, 3, 5, 10.0, seed=4)
    ref1 = ctx1.pnop_energy(u1)
    ref2 = ctx2.pnop_energy(u2)
    e1 = L.pnop_energy_noalloc(u1, W1, ctx1.nr, ctx1.M, ctx1.K, ctx1.Lz)
    e2 = L.pnop_energy_noalloc(u2, W2, ctx2.nr, ctx2.M, ctx2.K, ctx2.Lz)
    assert abs(e1 / ref1 - 1) < TOL
    assert abs(e2 / ref2 - 1) < TOL
    # and once more on the first field, after the small call
    e1b = L.pnop_energy_noalloc(u1, W1, ctx1.nr, ctx1.M, ctx1.K, ctx1.Lz)
    assert abs(e1b / ref1 - 1) < TOL
    ctx1.close()
    ctx2.close()


def test_noalloc_energy_rejects_fields_beyond_its_scratch(L):
    import torch
    u = torch.zeros(16, dtype=torch.complex128, device="cuda")
    W = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 3 * 512 * 255 * 256 > 2^24 complex values: rejected before any device work
    with pytest.raises(L.PnopError) as e:
        L.pnop_energy_noalloc(u, W, 512, 127, 255, 10.0)
    assert e.value.code == -1


def test_noalloc_energy_at_its_largest_size_on_a_side_stream(L):
    # 3 * 64 * 1 * 87381 = 2^24 - 64 complex values: the largest field of this
    # shape the fixed scratch serves (one more k is rejected, see the host
    # ABI tests), reduced on a non-default stream and checked against numpy
    import torch
    nr, M, K, Lz = 64, 0, 87380, 7.0
    gen = torch.Generator(device="cpu").manual_seed(11)
    u_h = torch.randn((3, nr, 2 * M + 1, K + 1, 2), generator=gen, dtype=torch.float64)
    W_h = torch.rand(nr, generator=gen, dtype=torch.float64) + 0.1
    uc = u_h[..., 0].numpy() + 1j * u_h[..., 1].numpy()
    ck = np.full(K + 1, 2.0)
    ck[0] = 1.0
    ref = 0.5 * 2 * np.pi * Lz * np.sum(W_h.numpy()[None, :, None, None] * ck * np.abs(uc) ** 2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        u = torch.view_as_complex(u_h.to("cuda", non_blocking=False)).contiguous()
        W = W_h.to("cuda")
    s.synchronize()
    for _ in range(2):
        e = L.pnop_energy_noalloc(u, W, nr, M, K, Lz, stream=s.cuda_stream)
        assert abs(e / ref - 1) < TOL
