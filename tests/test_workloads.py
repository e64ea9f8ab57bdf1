"""The seeded input generators: Philox4x32-10 known answers, Box-Muller
statistics and the C60-like geometry."""
import numpy as np

from itp_workloads import (cubic, c60_like_potential, normal_states,
                           philox4x32_10, random_wells_problem, supported_dim,
                           truncated_icosahedron)


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Random123 distribution)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
        ((0xffffffff,) * 4, (0xffffffff,) * 2,
         (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
        ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
         (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
    ]
    for ctr, key, want in cases:
        got = philox4x32_10(np.array([ctr[0]], np.uint32), ctr[1], ctr[2], ctr[3], *key)
        assert tuple(int(x[0]) for x in got) == want


def test_normal_states_statistics_and_addressing():
    a = normal_states(3, 20000, seed=1234)
    assert abs(a.mean()) < 0.02 and abs(a.std() - 1.0) < 0.02
    # any state can be regenerated alone
    b = normal_states(1, 20000, seed=1234, first_state=2)
    assert np.array_equal(a[2], b[0])
    assert not np.array_equal(a[0], normal_states(1, 20000, seed=1235)[0])


def test_truncated_icosahedron_geometry():
    v = truncated_icosahedron(6.7)
    assert v.shape == (60, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 6.7)
    d = np.linalg.norm(v[:, None] - v[None], axis=2) + np.eye(60) * 1e9
    nn = d.min(axis=1)
    # every vertex has 3 nearest neighbours at the common edge length
    assert np.allclose(nn, nn[0])
    assert all((np.abs(d[i] - nn[0]) < 1e-9).sum() == 3 for i in range(60))
    assert abs(nn[0] - 2.0 * 6.7 / np.sqrt(1 + 9 * ((1 + 5 ** 0.5) / 2) ** 2)) < 1e-9


def test_c60_like_depth():
    g = cubic(32, 32.0)
    V = c60_like_potential(g)
    assert V.max() <= 0.0 and -2.5 < V.min() < -1.5


def test_random_wells_problem_reproducible():
    g1, V1, n1 = random_wells_problem(1000, 5)
    g2, V2, n2 = random_wells_problem(1000, 5)
    assert g1 == g2 and n1 == n2 and np.array_equal(V1, V2)
    assert g1.nx in (32, 48, 64, 96) and 8 <= n1 <= 64


def test_supported_dims():
    for n in (2, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256):
        assert supported_dim(n)
    for n in (3, 5, 10, 54, 100, 512):
        assert not supported_dim(n)


def test_native_generator_matches_numpy():
    import itp_workloads as W
    W.build_native()
    a = W.normal_states(2, 4096, seed=77, problem=3, use_native=True)
    b = W.normal_states(2, 4096, seed=77, problem=3, use_native=False)
    assert np.array_equal(a, b)


def test_quantum_dot_array_geometry():
    from itp_workloads import planar, quantum_dot_array
    g = planar(128, 128, 32.0, 32.0)
    V = quantum_dot_array(g)
    assert V.shape == (1, 128, 128)
    # mirror symmetric about the box centre (grid point 64 is x = 0)
    core = V[0, 1:, 1:]
    np.testing.assert_allclose(core, core[::-1, :], atol=1e-12)
    np.testing.assert_allclose(core, core[:, ::-1], atol=1e-12)
    # the deepest points sit at dot centres: about -depth, plus the tails of
    # the neighbours (sech decays as 2 exp(-r/w))
    assert -2.2 < V.min() < -2.0
