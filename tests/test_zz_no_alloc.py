"""The allocation-free slice update (afqmc_update_slice_noalloc) against the
handle-based afqmc_update_slice.

Some callers cannot allocate device memory (they run inside another
framework's allocator or under a no-allocation policy), so the library offers
one entry point whose scratch lives in a static device array; the caller
brings only its G and field buffers.  Here both entry points update the same
G and field, twice in a row, and must agree: fields and accepted counts
exactly, G within the FP64 parity tolerance of the other GPU tests.  This file
is collected last on purpose."""
import numpy as np
import pytest

from synth import random_field

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as pkg
    return torch, pkg


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("L,beta,n_delay,n_stab", [(6, 1.0, 8, 5), (24, 1.6, 64, 8)])
def test_noalloc_matches_handle_update(env, L, beta, n_delay, n_stab):
    torch, pkg = env
    dtau, U, seed, chain = 0.1, 3.73, 91, 2
    ch = pkg.Chain(pkg.make_params(L=L, beta=beta, dtau=dtau, U=U, n_delay=n_delay, n_stab=n_stab,
                                   seed=seed, chain=chain))
    N, M = ch.N, ch.M
    assert N <= pkg.NOALLOC_MAX_N
    f = random_field(M, N, 555 + L)
    ch.set_field(f)
    G = ch.green(1)
    # caller-owned device buffers; the entry point itself allocates nothing
    G_dev = torch.from_numpy(G.copy()).to("cuda")
    s_dev = torch.from_numpy(f.copy()).to("cuda")
    stream = torch.cuda.current_stream()
    G_ref = G.copy()
    for call, (slice_, pas, sweep) in enumerate([(1, 0, 0), (1, 1, 3)]):
        # handle-based reference: updates its own copy of the field of this slice
        G_ref, n_ref = pkg.afqmc_update_slice(ch.h, slice_, pas, sweep, G_ref)
        f_ref = ch.field()
        n = pkg.afqmc_update_slice_noalloc(G_dev.data_ptr(), s_dev[slice_ - 1].data_ptr(), N, M, slice_, pas,
                                           sweep, U, dtau, n_delay, seed, chain, stream.cuda_stream)
        assert n == n_ref > 0, (call, n, n_ref)
        assert np.array_equal(s_dev.cpu().numpy()[slice_ - 1], f_ref[slice_ - 1]), call
        assert rel_err(G_dev.cpu().numpy(), G_ref) < TOL, call
    ch.close()


def test_noalloc_rejects_oversize(env):
    torch, pkg = env
    G_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    s_dev = torch.ones(4, dtype=torch.int8, device="cuda")
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_update_slice_noalloc(G_dev.data_ptr(), s_dev.data_ptr(), pkg.NOALLOC_MAX_N + 2, 10, 1, 0, 0,
                                       3.73, 0.1, 8, 1)
    assert e.value.code == 1 and "outside" in str(e.value)
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_update_slice_noalloc(G_dev.data_ptr(), s_dev.data_ptr(), 72, 10, 1, 0, 0,
                                       3.73, 0.1, pkg.NOALLOC_MAX_NDELAY + 1, 1)
    assert e.value.code == 1 and "n_delay" in str(e.value)
