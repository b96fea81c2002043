"""The allocation-free Gram product (samg_block_gram_noalloc) against the
allocating entry point (samg_block_gram): same kernels and summation order,
so the results must be bitwise equal, call after call."""
import pytest

pytestmark = pytest.mark.gpu


def _blocks(torch, rows, ld, seed):
    g = torch.Generator().manual_seed(seed)
    X = torch.randn(rows, ld, dtype=torch.float64, generator=g).cuda()
    Y = torch.randn(rows, ld, dtype=torch.float64, generator=g).cuda()
    return X, Y


@pytest.mark.parametrize("rows,nb,ld", [(300001, 8, 8), (4097, 10, 12), (1, 3, 4)])
def test_noalloc_gram_matches_allocating_gram_on_consecutive_calls(rows, nb, ld):
    import torch

    import paper_1102_0919_gb300 as samg

    stream = torch.cuda.current_stream()
    for call in range(2):
        X, Y = _blocks(torch, rows, ld, seed=100 * nb + call)
        G_ref = torch.full((nb, nb), float("nan"), dtype=torch.float64, device="cuda")
        G = torch.full((nb, nb), float("nan"), dtype=torch.float64, device="cuda")
        samg.block_gram(X.data_ptr(), Y.data_ptr(), rows, nb, ld, G_ref.data_ptr(), stream)
        samg.block_gram_noalloc(X.data_ptr(), Y.data_ptr(), rows, nb, ld, G.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(G, G_ref), (call, (G - G_ref).abs().max().item())
        plain = X[:, :nb].T @ Y[:, :nb]
        assert torch.allclose(G, plain, rtol=1e-12, atol=1e-10 * rows ** 0.5), call


def test_noalloc_gram_rejects_more_rows_than_its_scratch():
    import torch

    import paper_1102_0919_gb300 as samg

    # ceil(rows / 2048) * 16 * 16 = 514 * 256 > 131072 partial sums; real
    # buffers of that size are passed, so nothing outside them is touched
    rows, nb = 4096 * 257, 16
    X, Y = _blocks(torch, rows, nb, seed=5)
    G = torch.zeros(nb, nb, dtype=torch.float64, device="cuda")
    with pytest.raises(samg.SamgError, match="fixed scratch"):
        samg.block_gram_noalloc(X.data_ptr(), Y.data_ptr(), rows, nb, nb, G.data_ptr())
    # the largest accepted size (512 chunks of 2048 rows) still works
    rows = 4096 * 256
    samg.block_gram_noalloc(X.data_ptr(), Y.data_ptr(), rows, nb, nb, G.data_ptr())
    torch.cuda.synchronize()
    assert torch.allclose(G, X[:rows].T @ Y[:rows], rtol=1e-12, atol=1e-7)
