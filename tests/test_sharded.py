"""States of one problem split over ranks (paper_0809_3739_gb300.sharded):
the partition, the exchange (all-gather of phi), the replicated
orthonormalisation and Ritz step, and the slicing, checked with two and
three gloo ranks on the CPU.  Each rank's arithmetic comes from the oracle
here (a backend with the interface of AbiBackend), so the sharded step must
reproduce the oracle's single-process step (Eqs. 3 and 4, Sec. III) on the
same start states."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_0809_3739_gb300.sharded import split_counts  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    from itp_workloads import Grid, gaussian_wells_potential, normal_states
    g = Grid(12, 8, 6, 9.0, 7.0, 6.0)
    V = gaussian_wells_potential(g, np.array([[0.5, 0.2, -0.3], [-1.0, 0.4, 0.6]]),
                                 [2.0, 1.5], [0.9, 0.7])
    psi = normal_states(5, g.n_points, seed=808)
    return g, V, psi


class OracleBackend:
    """The ShardedStep backend interface with the oracle's arithmetic."""

    def __init__(self, g, V):
        from oracle import itp_oracle as O
        self.O, self.g, self.V = O, g, V
        self.psi = None

    def set_states(self, psi_local):
        self.psi = np.array(psi_local, dtype=np.float64, copy=True)

    def propagate(self, order, tau):
        return self.O.propagate(self.psi, self.V, self.g, order, tau)

    def orthonormalize(self, phi):
        return self.O.cholesky_orthonormalize(phi, self.g.dV)[0]

    def diagonal_energies(self, psi_local):
        return self.O.energies(psi_local, self.V, self.g, ritz=False)[0]

    def ritz(self, psi):
        E, rotated, _ = self.O.energies(psi, self.V, self.g, ritz=True)
        return E, rotated


def _worker(rank, world, port, ritz, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_0809_3739_gb300.sharded import ShardedStep
    g, V, psi = _problem()
    st = ShardedStep(OracleBackend(g, V), psi.shape[0])
    st.set_states(psi)
    out = []
    for _ in range(2):
        E, psi_local = st.step(6, 0.3, ritz=ritz)
        out.append((E, st.gather_states(psi_local), psi_local.shape[0]))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("ritz", [False, True])
def test_sharded_steps_equal_the_single_process_steps(world, ritz):
    from oracle import itp_oracle as O
    g, V, psi = _problem()
    ref = []
    p = psi
    for _ in range(2):
        p, E = O.itp_step(p, V, g, 6, 0.3, ritz=ritz)
        ref.append((E, p))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ritz, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = dict(q.get(timeout=180) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    counts = split_counts(psi.shape[0], world)
    for rank in range(world):
        for (E, states, m_local), (E_ref, p_ref) in zip(results[rank], ref):
            assert m_local == counts[rank]
            np.testing.assert_allclose(E, E_ref, rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(states, p_ref, rtol=0, atol=1e-11 * np.abs(p_ref).max())


def test_split_counts():
    assert split_counts(5, 2) == [3, 2]
    assert split_counts(5, 3) == [2, 2, 1]
    assert split_counts(128, 8) == [16] * 8
    assert split_counts(3, 4) == [1, 1, 1, 0]
    assert sum(split_counts(257, 7)) == 257
    with pytest.raises(ValueError):
        split_counts(0, 2)


def test_single_process_needs_no_group():
    from oracle import itp_oracle as O
    from paper_0809_3739_gb300.sharded import ShardedStep
    g, V, psi = _problem()
    st = ShardedStep(OracleBackend(g, V), psi.shape[0])
    assert (st.rank, st.world, st.s0, st.s1) == (0, 1, 0, psi.shape[0])
    st.set_states(psi)
    E, p = st.step(4, 0.2, ritz=True)
    p_ref, E_ref = O.itp_step(psi, V, g, 4, 0.2, ritz=True)
    np.testing.assert_allclose(E, E_ref, rtol=1e-13)
    np.testing.assert_allclose(p, p_ref, rtol=0, atol=1e-12)
