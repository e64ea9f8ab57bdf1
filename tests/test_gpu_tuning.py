"""Launch shapes (itp_set_tuning) and the autotuner (itp_autotune).

Every shape the autotuner may pick must give the oracle's results: each
valid combination of plane-pass form and pencil width is forced in turn and
checked against the oracle, on grids with ragged pencil blocks.
"""
import numpy as np
import pytest

from itp_workloads import Grid
from oracle import itp_oracle as O

from gpu_helpers import propagate_tolerance, report, seeded_states, wells_problem

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402

PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}
RB = {"fp64": 8, "mixed": 4}


def _relerr(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _row_pitch(nx):
    p = nx + nx // 16 + 2
    return p if p % 2 else p + 1


def _forms(g, prec):
    """(split, row_tb) pairs valid for the grid (the rules of itp.h)."""
    rb = RB[prec]
    whole_bytes = ((g.ny // 2) * _row_pitch(g.nx) + g.nx + g.ny) * 2 * rb
    out = [(0, 0)] if whole_bytes <= 227 * 1024 else []
    for tb in (32, 16, 8):
        if ((g.ny // 2) % tb == 0 and (tb * _row_pitch(g.nx) + g.nx) * 2 * rb <= 96 * 1024
                and (tb != 32 or (prec == "mixed" and g.nx == 256))):
            out.append((1, tb))
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("dims", [(64, 64, 8), (48, 32, 12)])
def test_every_launch_shape_matches_oracle(prec, dims):
    nx, ny, nz = dims
    g = Grid(nx, ny, nz, 14.0, 12.0, 6.0)
    V = wells_problem(g)
    m = 3
    psi = seeded_states(g, m)
    order, tau = 6, 0.3
    ref = O.propagate(psi, V, g, order, tau)
    psi_ref, _ = O.cholesky_orthonormalize(ref, g.dV)
    nxh = nx // 2 + 1
    widths = sorted({-(-nxh // c) for c in (1, 2, 3)})
    tol = propagate_tolerance(order, g.n_points, prec)
    with P.ItpGrid(nx, ny, nz, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as h:
        h.set_potential(V)
        base = h.get_tuning()
        for split, tb in _forms(g, prec):
            for w in widths:
                for ctas in (base["gram_ctas"], 7):
                    h.set_tuning(w, split, tb, ctas)
                    assert h.get_tuning() == {"pencil_w": w, "split": split, "row_tb": tb,
                                              "gram_ctas": ctas}
                    h.set_states(psi)
                    h.propagate(order, tau)
                    phi = h.get_phi()
                    report(f"{nx}x{ny}x{nz} {prec} propagate order {order} split={split} "
                           f"tb={tb} w={w}", _relerr(phi, ref), tol)
                    assert _relerr(phi, ref) < tol, (split, tb, w)
                    h.orthonormalize()
                    got = h.get_states()
                    assert _relerr(got, psi_ref) < (1e-11 if prec == "fp64" else 2e-4), \
                        (split, tb, w, ctas)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_autotune_keeps_states_and_results(prec):
    g = Grid(64, 64, 16, 14.0, 14.0, 8.0)
    V = wells_problem(g)
    m = 6
    psi = seeded_states(g, m)
    with P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as a, \
            P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as b:
        for h in (a, b):
            h.set_potential(V)
            h.set_states(psi)
        before = a.get_states()
        chosen, report = a.autotune(8, 0.25)
        assert np.array_equal(a.get_states(), before)
        assert a.get_tuning() == chosen
        for key in ("planes:", "pencil_w:", "gram:"):
            assert key in report, report
        for _ in range(3):
            Ea = a.step_graph(8, 0.25)
            Eb = b.step_graph(8, 0.25)
            assert np.max(np.abs(Ea - Eb)) < (1e-12 if prec == "fp64" else 1e-5) * np.max(np.abs(Eb))


def test_set_tuning_rejects_invalid_shapes():
    with P.ItpGrid(256, 256, 4, 20.0, 20.0, 4.0, 2, 0, P.ITP_MIXED) as h:
        base = h.get_tuning()
        assert base["split"] == 1   # a 256 x 256 FP32 plane does not fit one CTA
        bad = [dict(base, split=0),                 # must split
               dict(base, pencil_w=0), dict(base, pencil_w=130),
               dict(base, row_tb=12), dict(base, gram_ctas=0), dict(base, gram_ctas=10 ** 6)]
        for t in bad:
            with pytest.raises(P.ItpError) as ei:
                h.set_tuning(t["pencil_w"], t["split"], t["row_tb"], t["gram_ctas"])
            assert ei.value.code == P.itp.ITP_ERR_ARG
            assert h.get_tuning() == base


def test_batch_recaptures_after_a_shape_change():
    g = Grid(32, 32, 32, 12.0, 12.0, 12.0)
    V = wells_problem(g)
    psi = seeded_states(g, 4)
    with P.ItpBatch([(32, 32, 32)] * 2, [(12.0,) * 3] * 2, [4, 4], precision=P.ITP_FP64) as b:
        for q in b.problems:
            q.set_potential(V)
            q.set_states(psi)
        E0 = b.step(4, 0.2)
        n0 = b.kernel_launches
        t = b[1].get_tuning()
        b[1].set_tuning(9, 1, 8, t["gram_ctas"])   # split planes: more launches per step
        E1 = b.step(4, 0.2)
        assert b.kernel_launches - n0 > n0
        assert np.max(np.abs(E1[0] - E1[1])) < 1e-12 * np.max(np.abs(E1[0]))
        assert np.all(np.isfinite(E0[0]))


@pytest.mark.parametrize("form", [2, 3])
@pytest.mark.parametrize("dims", [(256, 256, 4), (256, 256, 1)])
def test_cluster_planes_match_oracle(dims, form):
    """256 x 256 FP32 planes on two- and four-CTA clusters (plane forms 2,
    3): propagation, orthonormalisation and Ritz values against the oracle,
    3D and planar."""
    from itp_workloads import planar
    nx, ny, nz = dims
    g = Grid(nx, ny, nz, 20.0, 18.0, 6.0) if nz > 1 else planar(nx, ny, 20.0, 18.0)
    V = wells_problem(g)
    m = 3
    psi = seeded_states(g, m)
    order, tau = 6, 0.3
    with P.ItpGrid(nx, ny, nz, g.lx, g.ly, g.lz, m, 0, P.ITP_MIXED) as h:
        h.set_potential(V)
        t = h.get_tuning()
        h.set_tuning(t["pencil_w"], form, 0, t["gram_ctas"])
        assert h.get_tuning()["split"] == form
        h.set_states(psi)
        h.propagate(order, tau)
        phi = h.get_phi()
        h.orthonormalize()
        E = h.energies("values")
    ref = O.propagate(psi, V, g, order, tau)
    report(f"{nx}x{ny}x{nz} mixed propagate order {order} cluster form {form}",
           _relerr(phi, ref), propagate_tolerance(order, g.n_points, "mixed"))
    assert _relerr(phi, ref) < propagate_tolerance(order, g.n_points, "mixed")
    psi_ref, _ = O.cholesky_orthonormalize(ref, g.dV)
    E_ref, _, _ = O.energies(psi_ref, V, g, ritz=True)
    assert np.max(np.abs(E - E_ref)) < 1e-5 * np.max(np.abs(E_ref))


def test_cluster_planes_only_where_they_apply():
    with P.ItpGrid(256, 256, 4, 20.0, 20.0, 4.0, 2, 0, P.ITP_FP64) as h:
        t = h.get_tuning()
        with pytest.raises(P.ItpError):
            h.set_tuning(t["pencil_w"], 2, 0, t["gram_ctas"])   # FP64 lane
    with P.ItpGrid(128, 128, 4, 20.0, 20.0, 4.0, 2, 0, P.ITP_MIXED) as h:
        t = h.get_tuning()
        with pytest.raises(P.ItpError):
            h.set_tuning(t["pencil_w"], 2, 0, t["gram_ctas"])   # not 256 x 256
        with pytest.raises(P.ItpError):
            h.set_tuning(t["pencil_w"], 3, 0, t["gram_ctas"])   # not 256 x 256
        with pytest.raises(P.ItpError):
            h.set_tuning(t["pencil_w"], 4, 0, t["gram_ctas"])
