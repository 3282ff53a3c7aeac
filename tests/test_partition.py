"""Element partitions of a sharded condensed operator (host logic of the library, CPU only):
the slab partition, the halo lists against the oracle's sparsity, and the two-exchange
operator application over world-size-2 gloo ranks against the oracle's S (Sec. 2.2,
eq. SC_step1)."""
import os
import socket

import numpy as np
import pytest

import oracle as O
import sc_inputs as I


def _system(n=4, N=2):
    Q, dt = I.tgv_state(n, N, cfl=10.0, seed=3)
    p = O.Params(n=n, N=N, dt=dt)
    return O.condensed_operator(O.jacobian(p, Q), n, N)


@pytest.mark.parametrize("n,nparts", [(4, 2), (4, 4), (5, 3)])
def test_slabs_give_every_element_one_rank(n, nparts):
    from paper_1911_02366_gb300 import sc
    part = sc.sc_partition_slabs(n, nparts)
    assert part.shape == (n ** 3,) and set(part.tolist()) == set(range(nparts))
    z = np.arange(n ** 3) // (n * n)
    for r in range(nparts):  # whole z-planes, contiguous
        planes = np.unique(z[part == r])
        assert np.all(np.diff(planes) == 1)
    owned = [sc.sc_partition_halo(n, part, r)[0] for r in range(nparts)]
    assert np.array_equal(np.sort(np.concatenate(owned)), np.arange(n ** 3))


def test_partition_rejects_bad_arguments():
    from paper_1911_02366_gb300 import sc
    for n, k in ((4, 0), (4, 5), (0, 1), (33, 2)):
        with pytest.raises(sc.SCError):
            sc.sc_partition_slabs(n, k)


@pytest.mark.parametrize("nparts", [2, 4])
def test_halo_lists_are_the_column_elements_of_the_owned_rows(nparts):
    """The owned rows of A_ib and A_bb reach boundary values exactly of owned + halo_b, the
    owned rows of A_bi interior values exactly of owned + halo_u."""
    from paper_1911_02366_gb300 import sc
    n, N = 4, 2
    cs = _system(n, N)
    ni, nb = cs.ni, cs.nb
    part = sc.sc_partition_slabs(n, nparts)
    for r in range(nparts):
        owned, hb, hu = sc.sc_partition_halo(n, part, r)
        own = set(owned.tolist())
        rows_i = np.concatenate([np.arange(e * ni, (e + 1) * ni) for e in owned])
        rows_b = np.concatenate([np.arange(e * nb, (e + 1) * nb) for e in owned])
        cols_b = set((cs.A_ib[rows_i].nonzero()[1] // nb).tolist()) | set((cs.A_bb[rows_b].nonzero()[1] // nb).tolist())
        cols_u = set((cs.A_bi[rows_b].nonzero()[1] // ni).tolist())
        assert cols_b - own == set(hb.tolist()), r
        assert cols_u - own == set(hu.tolist()), r


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port):
    import torch.distributed as dist
    from paper_1911_02366_gb300 import sc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, N = 4, 2
        cs = _system(n, N)
        ni, nb = cs.ni, cs.nb
        part = sc.sc_partition_slabs(n, world)
        lists = [sc.sc_partition_halo(n, part, r) for r in range(world)]
        owned, hb, hu = lists[rank]
        x = np.random.default_rng(11).standard_normal(n ** 3 * nb)  # the same global vector on every rank

        def exchange(vals, width, need):
            # every rank sends the blocks of its owned elements that another rank's list names
            mine = {int(e): vals[e * width:(e + 1) * width] for e in owned}
            outs = [None] * world
            dist.all_gather_object(outs, mine)
            got = {}
            for r, d in enumerate(outs):
                if r != rank:
                    got.update({e: v for e, v in d.items() if e in need})
            return got

        xl = np.zeros_like(x)  # owned values plus the received halo, zero elsewhere
        for e in owned:
            xl[e * nb:(e + 1) * nb] = x[e * nb:(e + 1) * nb]
        got = exchange(x, nb, set(hb.tolist()))
        assert set(got) == set(hb.tolist())
        for e, v in got.items():
            xl[e * nb:(e + 1) * nb] = v
        u = cs.aii_solve(cs.A_ib @ xl)  # valid on the owned elements (A_ii is block diagonal)
        ul = np.zeros_like(u)
        for e in owned:
            ul[e * ni:(e + 1) * ni] = u[e * ni:(e + 1) * ni]
        got = exchange(u, ni, set(hu.tolist()))
        assert set(got) == set(hu.tolist())
        for e, v in got.items():
            ul[e * ni:(e + 1) * ni] = v
        y = cs.A_bb @ xl - cs.A_bi @ ul
        ref = cs.matvec(x)
        rows = np.concatenate([np.arange(e * nb, (e + 1) * nb) for e in owned])
        assert np.max(np.abs(y[rows] - ref[rows])) <= 1e-12 * np.max(np.abs(ref)), rank
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_operator_over_two_gloo_ranks_equals_the_oracle():
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)
