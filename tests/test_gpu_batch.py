"""Batched chains (one CUDA graph per batched sweep), the slice kernel's grid
knob and the autotuner: all of them change only how the work is scheduled, so
every chain must end exactly where the same chain swept alone ends, and where
the CPU oracle's chain with the same seed ends."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


def mixed_params(pkg):
    mk = pkg.make_params
    return [mk(L=2, beta=1.0, dtau=0.1, U=3.73, n_delay=4, n_stab=5, seed=11, chain=0, measure=1, theta=(0.25, 0.5)),
            mk(L=3, beta=2.0, dtau=0.1, U=3.73, n_delay=4, n_stab=10, seed=12, chain=1, measure=1),
            mk(L=3, beta=1.0, dtau=0.1, U=3.0, n_delay=8, n_stab=5, seed=13, chain=2, measure=1, theta=(0.75, 0.25)),
            mk(L=6, beta=1.0, dtau=0.1, U=4.5, n_delay=16, n_stab=10, seed=14, chain=3, measure=1, update_ctas=9)]


def test_batch_equals_individual_chains(pkg):
    ps = mixed_params(pkg)
    batch = pkg.Batch(ps)
    st = batch.sweep(2)
    singles = [pkg.Chain(p) for p in ps]
    acc = 0
    for c in singles:
        acc += c.sweep(2).accepted
    assert st.accepted == acc > 0
    assert st.proposed == sum(2 * 2 * c.N * c.M for c in singles)
    assert st.launches > 0
    for cb, cs in zip(batch.chains, singles):
        assert np.array_equal(cb.field(), cs.field())
        gb, gs = cb.green(0), cs.green(0)
        assert np.abs(gb - gs).max() <= 1e-12 * np.abs(gs).max()
        ob, os_ = cb.observables(), cs.observables()
        assert ob["n_samples"] == os_["n_samples"] > 0
        for k in ("energy", "double_occ", "S_af"):
            assert abs(ob[k] - os_[k]) <= 1e-12 * max(1.0, abs(os_[k])), k
    # a second batched sweep replays the captured graph with the next sweep number
    batch.sweep(1)
    for c in singles:
        c.sweep(1)
    for cb, cs in zip(batch.chains, singles):
        assert np.array_equal(cb.field(), cs.field())
    for c in singles:
        c.close()
    batch.close()


def test_batch_chains_follow_the_oracle_in_lockstep(pkg):
    """Every chain of the mixed batch (periodic and twisted, L = 2..6, uneven
    n_delay and slice-kernel grids) against the CPU oracle's chain with the same
    seed: after each of two batched sweeps the fields are equal and G at slice 0
    agrees to 1e-10 (relative), with the same number of accepted flips."""
    from oracle.dqmc import Model, Chain
    ps = mixed_params(pkg)
    batch = pkg.Batch(ps)
    oracles = [Chain(Model(p.L1, U=p.U, beta=p.beta, dtau=p.dtau, theta=(p.theta1, p.theta2)),
                     n_delay=p.n_delay, n_stab=p.n_stab, seed=p.seed, chain=p.chain) for p in ps]
    for cb, oc in zip(batch.chains, oracles):
        assert np.array_equal(cb.field(), oc.field)
    for _ in range(2):
        acc0 = [oc.accepted for oc in oracles]
        st = batch.sweep(1)
        for oc in oracles:
            oc.sweep()
        assert st.accepted == sum(oc.accepted - a for oc, a in zip(oracles, acc0)) > 0
        for cb, oc in zip(batch.chains, oracles):
            assert np.array_equal(cb.field(), oc.field)
            g = cb.green(0)
            assert np.abs(g - oc.G).max() <= 1e-10 * np.abs(oc.G).max()
    batch.close()


def test_update_grid_does_not_change_the_chain(pkg):
    ps = [pkg.make_params(L=6, beta=1.0, dtau=0.1, U=3.73, n_delay=16, n_stab=5, seed=5, update_ctas=g)
          for g in (0, 5, 37)]
    chains = [pkg.Chain(p) for p in ps]
    for c in chains:
        c.sweep(1)
    f0, g0 = chains[0].field(), chains[0].green(0)
    for c in chains[1:]:
        assert np.array_equal(c.field(), f0)
        assert np.abs(c.green(0) - g0).max() <= 1e-12 * np.abs(g0).max()
    for c in chains:
        c.close()


def test_autotune_picks_a_candidate(pkg):
    ps = [pkg.make_params(L=3, beta=1.0, dtau=0.1, U=3.73, n_delay=4, n_stab=5, seed=s, chain=s, theta=th)
          for s, th in enumerate([(0.0, 0.0), (0.25, 0.0), (0.5, 0.5), (0.75, 0.25)])]
    nd, ct, rate = pkg.afqmc_batch_autotune(ps, [2, 8], [0, 6], n_timed=1)
    assert nd in (2, 8) and ct in (0, 6) and rate > 0
    with pytest.raises(pkg.AfqmcError):
        pkg.afqmc_batch_autotune(ps, [], [0])
