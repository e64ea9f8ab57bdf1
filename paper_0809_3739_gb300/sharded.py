"""The states of one problem split over the ranks of a torch.distributed
process group.

Sec. IV of the paper distributes the states over processors: the
propagation of Eq. (3) acts on each state alone, and only the
orthonormalisation of Eq. (4) (and the subspace matrix of the Ritz step,
Sec. III) couples them.  Rank r of W holds the states [s_r, s_r+1) of an
even split in the global order (the first m % W ranks one more).  One step:

  1. phi_j = T_2k(tau) psi_j for the rank's own states, no exchange;
  2. the exchange: an all-gather of phi, so every rank holds the m x N block;
  3. psi = L^{-1} phi with S = phi phi^T dV = L L^T, replicated on every rank;
  4. energies: without the Ritz step the diagonal (psi_j|H|psi_j) dV of the
     rank's own states, gathered; with it the eigenvalues of the whole
     subspace matrix and the rotation of the block onto its eigenvectors,
     replicated;
  5. the rank keeps its slice of psi.

The module partitions, exchanges and slices; each stage's arithmetic is a
backend's.  `AbiBackend` runs it in this library's kernels on the rank's GPU
(the local propagation on an ItpGrid of the rank's states, the replicated
orthonormalisation by itp_orthonormalize_noalloc, the Ritz step on an ItpGrid
of all m states).  The exchange goes through the process group: CUDA
tensors under NCCL, host tensors otherwise.
"""
import numpy as np


def split_counts(m, world):
    """States per rank: an even split, the first m % world ranks one more."""
    if m < 1 or world < 1:
        raise ValueError("need m >= 1 states and world >= 1 ranks")
    base, extra = divmod(m, world)
    return [base + (1 if r < extra else 0) for r in range(world)]


def _dist():
    import torch.distributed as dist
    return dist


def _group_info(group):
    dist = _dist()
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return 0, 1, False
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    nccl = dist.get_backend(group) == "nccl"
    return rank, world, nccl


def all_gather_rows(local, counts, group=None):
    """The rows of every rank's `local` (shape (counts[rank], n)), in rank
    order, on every rank: an all-gather of blocks padded to max(counts)
    rows."""
    import torch
    rank, world, nccl = _group_info(group)
    local = np.ascontiguousarray(local, dtype=np.float64)
    if world == 1:
        return local.copy()
    if local.shape[0] != counts[rank]:
        raise ValueError("local block has %d rows, the split gives %d" %
                         (local.shape[0], counts[rank]))
    rows = max(counts)
    n = local.shape[1]
    device = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")
    send = torch.zeros((rows, n), dtype=torch.float64, device=device)
    send[:local.shape[0]] = torch.from_numpy(local).to(device)
    recv = [torch.empty_like(send) for _ in range(world)]
    _dist().all_gather(recv, send, group=group)
    return np.concatenate([recv[r][:counts[r]].cpu().numpy() for r in range(world)], axis=0)


class ShardedStep:
    """One problem's m states over the ranks of `group` (None: the default
    process group, or a single process without one).  `backend` supplies
    the arithmetic (see AbiBackend for the interface)."""

    def __init__(self, backend, m, group=None):
        self.backend = backend
        self.group = group
        self.rank, self.world, _ = _group_info(group)
        if m < self.world:
            raise ValueError("%d states cannot give each of %d ranks one" % (m, self.world))
        self.counts = split_counts(m, self.world)
        self.m = m
        self.s0 = sum(self.counts[:self.rank])
        self.s1 = self.s0 + self.counts[self.rank]

    def set_states(self, psi_all):
        """Hand the rank its slice of the m x N start block (every rank
        passes the same block)."""
        psi_all = np.asarray(psi_all, dtype=np.float64)
        if psi_all.shape[0] != self.m:
            raise ValueError("expected %d states, got %d" % (self.m, psi_all.shape[0]))
        self.backend.set_states(psi_all[self.s0:self.s1])

    def step(self, order, tau, ritz=False):
        """One step; returns (E, psi_local): all m energies (the same on
        every rank) and the rank's own orthonormal states."""
        phi_local = self.backend.propagate(order, tau)
        phi = all_gather_rows(phi_local, self.counts, self.group)
        psi = self.backend.orthonormalize(phi)
        if ritz:
            E, psi = self.backend.ritz(psi)
            psi_local = psi[self.s0:self.s1]
        else:
            psi_local = psi[self.s0:self.s1]
            E_local = self.backend.diagonal_energies(psi_local)
            E = all_gather_rows(np.asarray(E_local, dtype=np.float64)[:, None], self.counts,
                                self.group)[:, 0]
        self.backend.set_states(psi_local)
        return np.asarray(E), psi_local

    def gather_states(self, psi_local):
        """The m x N block of all ranks' states, on every rank."""
        return all_gather_rows(psi_local, self.counts, self.group)


class AbiBackend:
    """The arithmetic of a ShardedStep in this library's kernels on the
    current GPU.  dims = (nx, ny, nz), box = (lx, ly, lz); V the potential
    [nz][ny][nx] (Hartree); m_local the rank's states, m the problem's.

    Interface used by ShardedStep:
      set_states(psi_local)        the rank's states (host float64 rows)
      propagate(order, tau)        -> phi_local (host float64 rows), Eq. (3)
      orthonormalize(phi)          -> psi for the whole block (FP64), Eq. (4)
      diagonal_energies(psi_local) -> (psi_j|H|psi_j) dV of the rank's states
      ritz(psi)                    -> (E, psi rotated), the Ritz step of Sec. III
    """

    def __init__(self, dims, box, V, m_local, m, precision=None):
        import paper_0809_3739_gb300 as P
        self._P = P
        nx, ny, nz = dims
        lx, ly, lz = box
        prec = P.ITP_FP64 if precision is None else precision
        if m > 128:
            raise ValueError("the replicated orthonormalisation takes m <= 128 states")
        self.n_points = nx * ny * nz
        self.dV = lx * ly * lz / self.n_points
        self.m = m
        self.local = P.ItpGrid(nx, ny, nz, lx, ly, lz, m_local, 0, prec)
        self.local.set_potential(V)
        self.full = P.ItpGrid(nx, ny, nz, lx, ly, lz, m, 0, prec)
        self.full.set_potential(V)

    def close(self):
        self.local.close()
        self.full.close()

    def set_states(self, psi_local):
        self.local.set_states(psi_local)

    def propagate(self, order, tau):
        self.local.propagate(order, tau)
        return self.local.get_phi()

    def orthonormalize(self, phi):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        src = torch.from_numpy(np.ascontiguousarray(phi, dtype=np.float64)).to(dev)
        dst = torch.empty_like(src)
        stream = torch.cuda.current_stream(dev)
        self._P.itp_orthonormalize_noalloc(src.data_ptr(), dst.data_ptr(), self.m,
                                           self.n_points, self.dV, stream.cuda_stream)
        return dst.cpu().numpy()

    def diagonal_energies(self, psi_local):
        self.local.set_states(psi_local)
        return self.local.energies(False)

    def ritz(self, psi):
        self.full.set_states(psi)
        E = self.full.energies(True)
        return E, self.full.get_states()
