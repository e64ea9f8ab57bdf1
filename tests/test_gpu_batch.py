"""Batches of independent problems (itp_create_batch / itp_batch_step).

A batch step is every problem's itp_step, captured as parallel branches of
one CUDA graph.  The problems come from the seeded random-well generator of
the batched workload (uneven grids and state counts).
"""
import numpy as np
import pytest

from itp_workloads import normal_states, random_wells_problem
from oracle import itp_oracle as O

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402

PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}


def _problems(count, sizes, n_range, seed=1000):
    out = []
    for p in range(count):
        g, V, n = random_wells_problem(seed, p, sizes=sizes, n_range=n_range)
        out.append((g, V, normal_states(n, g.n_points, seed, problem=p)))
    return out


def _batch(problems, prec):
    dims = [(g.nx, g.ny, g.nz) for g, _, _ in problems]
    boxes = [(g.lx, g.ly, g.lz) for g, _, _ in problems]
    ns = [psi.shape[0] for _, _, psi in problems]
    b = P.ItpBatch(dims, boxes, ns, precision=PREC[prec])
    for q, (g, V, psi) in zip(b.problems, problems):
        q.set_potential(V)
        q.set_states(psi)
    return b


@pytest.mark.parametrize("grouped", [True, False])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_equals_single_problem_steps(prec, grouped):
    """Every CTA of a batch step computes what the problem's own itp_step
    computes, whether the passes of problems with one grid run as grouped
    launches or each problem is its own graph branch: energies and states
    agree exactly.  The branch form launches as many kernels as the single
    steps together; the grouped form fewer."""
    problems = _problems(5, (32, 48, 64), (3, 8))
    singles = []
    for g, V, psi in problems:
        h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, psi.shape[0], 0, PREC[prec])
        h.set_potential(V)
        h.set_states(psi)
        singles.append(h)
    with _batch(problems, prec) as b:
        b.set_grouping(grouped)
        for step in range(3):
            Eb = b.step(8, 0.25)
            l0 = [h.kernel_launches for h in singles]
            Es = [h.step_graph(8, 0.25) for h in singles]
            for p in range(len(problems)):
                assert np.array_equal(Eb[p], Es[p]), (step, p)
            if step == 1:   # step 0 also built the tables, outside the graphs
                per_step = sum(h.kernel_launches - a for h, a in zip(singles, l0))
        if grouped:
            assert b.groups >= 1
            assert b.kernel_launches < 3 * per_step
        else:
            assert b.kernel_launches == 3 * per_step
        for q, h in zip(b.problems, singles):
            assert np.array_equal(q.get_states(), h.get_states())
    for h in singles:
        h.close()


def test_batch_fp64_matches_oracle():
    """Three 32^3 problems in FP64: two batch steps against the oracle's
    iterations (Ritz values; the oracle rotates, the batch does not, and the
    values depend only on the span)."""
    problems = _problems(3, (32,), (3, 8), seed=1100)
    refs = [psi.copy() for _, _, psi in problems]
    with _batch(problems, "fp64") as b:
        for _ in range(2):
            Eb = b.step(8, 0.25)
            for p, (g, V, _) in enumerate(problems):
                refs[p], E_ref = O.itp_step(refs[p], V, g, 8, 0.25)
                assert np.max(np.abs(Eb[p] - E_ref)) < 1e-11 * np.max(np.abs(E_ref)), p


def test_batch_mixed_then_fp64_steps_match_oracle():
    """Mixed problems: an FP32 step within the mixed tolerance of the oracle,
    then ITP_STEP_FP64 steps, which continue in FP64 from the FP32 states:
    the oracle, started from the same states rounded to FP32, matches them to
    FP64 accuracy."""
    problems = _problems(3, (32,), (3, 6), seed=1200)
    with _batch(problems, "mixed") as b:
        E32 = b.step(8, 0.25)
        for p, (g, V, psi) in enumerate(problems):
            _, E_ref = O.itp_step(psi, V, g, 8, 0.25)
            assert np.max(np.abs(E32[p] - E_ref)) < 1e-5 * np.max(np.abs(E_ref)), p
        # the states after the FP32 step are FP32 values; continue in FP64
        start = [q.get_states() for q in b.problems]
        E64 = [b.step(8, 0.25, fp64=True) for _ in range(2)]
        for p, (g, V, _) in enumerate(problems):
            ref = start[p]
            for s in range(2):
                ref, E_ref = O.itp_step(ref, V, g, 8, 0.25)
                assert np.max(np.abs(E64[s][p] - E_ref)) < 1e-11 * np.max(np.abs(E_ref)), (p, s)


def test_batch_errors_name_the_problem():
    with pytest.raises(P.ItpError) as ei:
        P.ItpBatch([(32, 32, 32), (32, 32, 32), (10, 32, 32)], [(16.0,) * 3] * 3, [4, 4, 4])
    assert ei.value.code == P.itp.ITP_ERR_ARG and "problem 2" in str(ei.value)
    problems = _problems(2, (32,), (3, 4), seed=1300)
    b = P.ItpBatch([(g.nx, g.ny, g.nz) for g, _, _ in problems],
                   [(g.lx, g.ly, g.lz) for g, _, _ in problems],
                   [psi.shape[0] for _, _, psi in problems], precision=P.ITP_MIXED)
    with b:
        g, V, psi = problems[0]
        b[0].set_potential(V)
        b[0].set_states(psi)
        b[1].set_states(problems[1][2])   # no potential on problem 1
        with pytest.raises(P.ItpError) as ei:
            b.step(4, 0.2)
        assert ei.value.code == P.itp.ITP_ERR_STATE and "problem 1" in str(ei.value)
        b[1].set_potential(problems[1][1])
        E = b.step(4, 0.2)   # usable after the error
        assert all(np.all(np.isfinite(e)) for e in E)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_grouped_batch_matches_branch_form(prec):
    """Twelve problems on three grids (several per grid, uneven state counts):
    grouped launches and the per-problem graph give the same energies and
    states bit for bit, step after step, also for FP64 steps of a mixed
    batch; three groups."""
    problems = _problems(12, (32, 48, 64), (2, 9), seed=1400)
    with _batch(problems, prec) as a, _batch(problems, prec) as c:
        c.set_grouping(False)
        for step in range(3):
            fp64 = prec == "mixed" and step == 2
            Ea = a.step(8, 0.25, fp64=fp64)
            Ec = c.step(8, 0.25, fp64=fp64)
            for p in range(len(problems)):
                assert np.array_equal(Ea[p], Ec[p]), (step, p)
        assert a.groups == 3 and c.groups == 0
        for qa, qc in zip(a.problems, c.problems):
            assert np.array_equal(qa.get_states(), qc.get_states())


def test_batch_with_tmem_pencils_equals_single_problem_steps():
    """Problems with nz = 128 whose pencil width is 0 (one thread per z
    column, the column in TMEM) take part in a grouped batch: their pencil
    passes run as per-problem launches (the TMEM pencil has no grouped
    form), the plane passes of the two problems on one grid as grouped
    launches; energies and states equal the problems' own graph steps with
    the same launch shapes, bit for bit."""
    from gpu_helpers import seeded_states, wells_problem
    from itp_workloads import Grid

    grids = [Grid(48, 24, 128, 14.0, 10.0, 40.0), Grid(48, 24, 128, 14.0, 10.0, 40.0),
             Grid(32, 32, 128, 12.0, 12.0, 40.0)]
    problems = [(g, wells_problem(g), seeded_states(g, 3 + p, seed=300 + p))
                for p, g in enumerate(grids)]
    singles = []
    for g, V, psi in problems:
        h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, psi.shape[0], 0, P.ITP_MIXED)
        h.set_potential(V)
        h.set_states(psi)
        t = h.get_tuning()
        h.set_tuning(0, t["split"], t["row_tb"], t["gram_ctas"])
        singles.append(h)
    with _batch(problems, "mixed") as b:
        for q in b.problems:
            t = q.get_tuning()
            q.set_tuning(0, t["split"], t["row_tb"], t["gram_ctas"])
        for step in range(2):
            Eb = b.step(8, 0.25)
            Es = [h.step_graph(8, 0.25) for h in singles]
            for p in range(len(problems)):
                assert np.array_equal(Eb[p], Es[p]), (step, p)
        for q, h in zip(b.problems, singles):
            assert np.array_equal(q.get_states(), h.get_states())
    for h in singles:
        h.close()
