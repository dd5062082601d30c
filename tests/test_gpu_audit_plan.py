"""The batched audit plan (rtt_audit_plan_*): all (geometry, arm) jobs of the
class-Gram audit in one launch per stage.

  * the twelve geometries at the paper's eight-frame sampling (uneven table
    sizes) in ONE plan, against the oracle's stored values (rank, L_anchor,
    J_old, A_{0,0.999}, sigma_max), as tests/test_gpu_audit12_golden.py
    checks them geometry by geometry;
  * the plan against the per-geometry entry points (probe information, reach,
    class Gram and its spectrum) on small geometries;
  * a run replayed twice, and replayed from a captured CUDA graph, gives the
    same records bit for bit.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "audit12_oracle.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rtt.lib()


def _optable(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


def _key(w):
    import sys
    p = os.path.join(HERE, "golden")
    if p not in sys.path:
        sys.path.insert(0, p)
    import make_audit12
    return make_audit12.workload_key(w)


def test_twelve_geometries_in_one_plan_match_the_oracle():
    with open(GOLDEN) as fh:
        data = json.load(fh)
    recs = {c["key"]: c for c in data["paper8"]["cells"]}
    cells = I.audit12_paper_sampling()
    ops, refs = [], []
    for w in cells:
        tab = O.build_table(w, I.screen_samples(w))
        ops.append(rtt.Operator(w, _optable(tab)))
        refs.append(recs[_key(w)])
    assert len({o.info.n_rays for o in ops}) > 1  # uneven tables
    plan = rtt.AuditPlan(ops, (1, 7))
    plan.run()
    out, sig = plan.results()
    for g, ref in enumerate(refs):
        for a, arm in enumerate(("direct", "resolved")):
            rec, r = out[g][a], ref["arms"][arm]
            if r["margin"] >= 1e-6:
                assert rec.rank == r["rank"], (ref["name"], arm, rec.rank, r["rank"])
            assert rec.reach.L_anchor == r["L_anchor"], (ref["name"], arm)
            assert abs(rec.reach.J_old - r["J_old"]) <= 1e-5 * max(r["J_old"], 1.0)
            assert abs(rec.reach.A0q - ref["A0999"]) <= 1e-12 * max(abs(ref["A0999"]), 1.0)
            assert rec.sigma_max == pytest.approx(r["sigma_max"], rel=1e-9)
    plan.close()
    for o in ops:
        o.close()


@pytest.fixture(scope="module")
def small_ops():
    ops = []
    for spin, incl, nx in ((0.0, 30.0, 40), (0.5, 50.0, 48), (0.94, 75.0, 36)):
        w = I.small_kerr(spin=spin, incl_deg=incl, nx=nx, n_r=10, n_phi=20, n_frames=120,
                         n_hats=40, ss=2)
        tab = O.build_table(w, I.screen_samples(w))
        ops.append(rtt.Operator(w, _optable(tab)))
    yield ops
    for o in ops:
        o.close()


def test_plan_matches_the_per_geometry_entry_points(small_ops):
    ages = rtt.AGES
    plan = rtt.AuditPlan(small_ops, (1, 7), ages=ages)
    plan.run()
    out, sig = plan.results()
    for g, op in enumerate(small_ops):
        a0 = rtt.direct_age_quantile(op, 0.999)
        for a, mask in enumerate((1, 7)):
            info = rtt.probe_info(op, mask, ages)
            res, _ = rtt.reach(op, info, mask, ages, a0q=a0, age_step=ages[1] - ages[0])
            rec = out[g][a]
            assert rec.reach.L_anchor == res.L_anchor and rec.reach.anchor_index == res.anchor_index
            assert rec.reach.J_old == pytest.approx(res.J_old, rel=1e-9)
            assert rec.reach.A0q == a0
            G = rtt.gram_class(op, rtt.CLASS_S224, mask)
            s_ref, rank, _ = rtt.rank_from_eigenvalues(np.linalg.eigvalsh(G.cpu().numpy()))
            assert rec.rank == rank
            np.testing.assert_allclose(sig[g, a], s_ref, rtol=1e-8, atol=1e-9 * s_ref[0])
    plan.close()


def _records(out):
    return [(r.rank, r.margin, r.sigma_max, r.reach.J_old, r.reach.L_anchor) for row in out for r in row]


def test_plan_replays_and_graph_capture_are_bitwise(small_ops):
    plan = rtt.AuditPlan(small_ops, (1, 7))
    plan.run()
    out1, sig1 = plan.results()
    plan.run()
    out2, sig2 = plan.results()
    assert _records(out1) == _records(out2) and np.array_equal(sig1, sig2)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        graph.capture_begin()
        plan.run(stream=s)
        graph.capture_end()
    graph.replay()
    torch.cuda.synchronize()
    out3, sig3 = plan.results(stream=s)
    assert _records(out3) == _records(out1) and np.array_equal(sig3, sig1)
    plan.close()
