"""Failure paths of the boundary, exercised without faulting the GPU.

* A device-side wait that runs out: the test hook afqmc_set_wait_limit shortens
  the limit of the waits between CTAs (grid barriers, QR/LU hand-offs) to 1 ns,
  so the first wait of the next sweep runs out; the kernel sets the handle's
  error flag and returns, the call reports AFQMC_E_TIMEOUT, the handle then
  refuses work (AFQMC_E_STATE), and the CUDA context stays usable (a new
  chain sweeps normally).
* A non-finite value in a host matrix handed to the test hooks: the slice
  update meets a NaN ratio and the wrap a NaN result; both report
  AFQMC_E_NUMERIC, then AFQMC_E_STATE.
Nothing here traps, faults or hangs the GPU: every wait is bounded, and the
poisoned values are host data."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

E_NUMERIC, E_TIMEOUT, E_STATE = 4, 5, 6


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


def small(pkg, **kw):
    return pkg.Chain(pkg.make_params(L=2, beta=1.0, dtau=0.1, U=3.73, n_delay=4, n_stab=5, seed=3, **kw))


def test_wait_that_runs_out_reports_timeout(pkg):
    ch = small(pkg)
    ch.sweep(1)                                   # default limit: fine
    pkg.afqmc_set_wait_limit(ch.h, 1)             # 1 ns: the next wait between CTAs runs out
    with pytest.raises(pkg.AfqmcError) as e:
        ch.sweep(1)
    assert e.value.code == E_TIMEOUT, e.value
    assert "timed out" in str(e.value)
    with pytest.raises(pkg.AfqmcError) as e:
        ch.sweep(1)
    assert e.value.code == E_STATE
    ch.close()
    fresh = small(pkg)                            # the context is still usable
    assert fresh.sweep(1).accepted > 0
    fresh.close()


def test_restoring_the_default_limit_keeps_the_chain_exact(pkg):
    a, b = small(pkg), small(pkg)
    pkg.afqmc_set_wait_limit(a.h, 0)              # 0 = the default limit
    a.sweep(2)
    b.sweep(2)
    assert np.array_equal(a.field(), b.field())
    a.close()
    b.close()


@pytest.mark.parametrize("theta", [(0.0, 0.0), (0.25, 0.5)])
def test_nan_in_host_green_function_of_slice_update(pkg, theta):
    ch = small(pkg, theta=theta)
    G = ch.green(1)
    G[0, 0] = np.nan
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_update_slice(ch.h, 1, 0, 0, G)
    assert e.value.code == E_NUMERIC, e.value
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_update_slice(ch.h, 1, 0, 0, np.eye(G.shape[0], dtype=G.dtype))
    assert e.value.code == E_STATE
    ch.close()


@pytest.mark.parametrize("direction", [+1, -1, 0])
def test_nan_in_host_matrix_of_wrap(pkg, direction):
    ch = small(pkg)
    A = ch.green(1)
    A[3, 5] = np.inf
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_wrap_matrix(ch.h, 1, direction, A)
    assert e.value.code == E_NUMERIC, e.value
    with pytest.raises(pkg.AfqmcError) as e:
        ch.sweep(1)
    assert e.value.code == E_STATE
    ch.close()
