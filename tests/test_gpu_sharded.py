"""The arithmetic backend of the sharded step (paper_0809_3739_gb300.sharded
.AbiBackend) on one GPU: the rank's propagation on an ItpGrid of its
states, the replicated orthonormalisation (itp_orthonormalize_noalloc) and
the Ritz step on an ItpGrid of all states, driven by ShardedStep in a single
process, against the oracle's steps (FP64 path).  The exchange itself is
checked on CPU gloo ranks (test_sharded.py) and, below, with two and three
ranks as processes sharing the GPU."""
import numpy as np
import pytest

from itp_workloads import Grid, gaussian_wells_potential, normal_states
from oracle import itp_oracle as O

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402,F401
from paper_0809_3739_gb300.sharded import AbiBackend, ShardedStep  # noqa: E402


@pytest.mark.parametrize("ritz", [False, True])
def test_abi_backend_steps_match_oracle(ritz):
    g = Grid(24, 16, 12, 9.0, 7.0, 6.0)
    V = gaussian_wells_potential(g, np.array([[0.5, 0.2, -0.3], [-1.0, 0.4, 0.6]]),
                                 [2.0, 1.5], [0.9, 0.7])
    m = 5
    psi = normal_states(m, g.n_points, seed=909)
    be = AbiBackend((g.nx, g.ny, g.nz), (g.lx, g.ly, g.lz), V, m, m)
    try:
        st = ShardedStep(be, m)
        st.set_states(psi)
        ref = psi
        for _ in range(2):
            E, p = st.step(6, 0.3, ritz=ritz)
            ref, E_ref = O.itp_step(ref, V, g, 6, 0.3, ritz=ritz)
            assert np.max(np.abs(E - E_ref)) < 1e-11 * np.max(np.abs(E_ref))
            if ritz:
                # Ritz vectors are unique up to sign (the eigenvalues here
                # are simple): compare after aligning each state's sign
                sign = np.sign(np.sum(p * ref, axis=1))
                p = p * sign[:, None]
            assert np.max(np.abs(p - ref)) < 1e-10 * np.max(np.abs(ref))
    finally:
        be.close()


# Two and three ranks in separate processes, each running its own kernels on
# the one visible GPU; the exchange is an all-gather of host buffers over
# gloo, so no kernel of one rank waits on another rank.
def _abi_problem():
    g = Grid(24, 16, 12, 9.0, 7.0, 6.0)
    V = gaussian_wells_potential(g, np.array([[0.5, 0.2, -0.3], [-1.0, 0.4, 0.6]]),
                                 [2.0, 1.5], [0.9, 0.7])
    psi = normal_states(5, g.n_points, seed=919)
    return g, V, psi


def _abi_worker(rank, world, port, ritz, q):
    import os
    import torch
    import torch.distributed as dist
    from paper_0809_3739_gb300.sharded import split_counts as counts_of
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, V, psi = _abi_problem()
    m = psi.shape[0]
    be = AbiBackend((g.nx, g.ny, g.nz), (g.lx, g.ly, g.lz), V, counts_of(m, world)[rank], m)
    out = []
    try:
        st = ShardedStep(be, m)
        st.set_states(psi)
        for _ in range(2):
            E, psi_local = st.step(6, 0.3, ritz=ritz)
            out.append((E, st.gather_states(psi_local), psi_local.shape[0]))
    finally:
        be.close()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("ritz", [False, True])
def test_ranks_in_processes_match_oracle(world, ritz):
    import socket
    import torch.multiprocessing as mp
    from paper_0809_3739_gb300.sharded import split_counts
    g, V, psi = _abi_problem()
    ref, p = [], psi
    for _ in range(2):
        p, E = O.itp_step(p, V, g, 6, 0.3, ritz=ritz)
        ref.append((E, p))
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_abi_worker, args=(r, world, port, ritz, q))
             for r in range(world)]
    for pr in procs:
        pr.start()
    try:
        results = dict(q.get(timeout=240) for _ in procs)
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
    assert all(pr.exitcode == 0 for pr in procs)
    counts = split_counts(psi.shape[0], world)
    for rank in range(world):
        for (E, states, m_local), (E_ref, p_ref) in zip(results[rank], ref):
            assert m_local == counts[rank]
            assert np.max(np.abs(E - E_ref)) < 1e-11 * np.max(np.abs(E_ref))
            if ritz:
                states = states * np.sign(np.sum(states * p_ref, axis=1))[:, None]
            assert np.max(np.abs(states - p_ref)) < 1e-10 * np.max(np.abs(p_ref))
