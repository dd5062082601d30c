"""The 12-geometry rank audit (Sec. 6.2-6.3) at full kerr256 sizes against the
FP64 oracle: rtt_rank_audit on the oracle's own ray tables, compared with the
values tests/golden/make_audit12.py wrote from the oracle alone (the
restricted S224 Gram formed as Q^T A^T A Q with the oracle's applies, its
eigenvalues, the probe information, reach and old-age innovation).

Operational rank and L_anchor must equal the oracle's (every cell's margin
is far above the FP64 resolution of the Gram; a cell with margin below 1e-6
would be parity unpinned and is skipped), J_old agrees to 1e-5 relative
(FP32 exponentials with FP64 reduction), A_{0,0.999} to 1e-12."""
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
sys_path = os.path.join(HERE, "golden")


def _key(w):
    import sys
    if sys_path not in sys.path:
        sys.path.insert(0, sys_path)
    import make_audit12
    return make_audit12.workload_key(w)


@pytest.mark.parametrize("sampling", ["paper8", "frames256"])
@pytest.mark.parametrize("mode", ["class", "normal"])
def test_rank_audit_matches_the_oracle(sampling, mode):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with open(GOLDEN) as fh:
        data = json.load(fh)
    if sampling not in data:
        pytest.skip(f"no oracle record for the {sampling} sampling")
    build.build()
    recs = {c["key"]: c for c in data[sampling]["cells"]}
    cells = I.audit12_paper_sampling() if sampling == "paper8" else I.audit12()
    gram_mode = rtt.GRAM_CLASS_S224 if mode == "class" else rtt.GRAM_NORMAL
    n_checked = 0
    for w in cells:
        ref = recs.get(_key(w))
        if ref is None:
            continue
        tab = O.build_table(w, I.screen_samples(w))
        assert tab.n_rays == ref["n_rays"] and tab.n_rows == ref["n_rows"]
        op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                              "delay": tab.delay, "weight": tab.weight,
                              "throughput": tab.throughput})
        Q = rtt.synth_class(op, rtt.CLASS_S224) if mode == "normal" else None
        out, _ = rtt.rank_audit([op], [Q], (1, 7), mode=gram_mode)
        for rec, arm in zip(out[0], ("direct", "resolved")):
            r = ref["arms"][arm]
            if r["margin"] >= 1e-6:
                assert rec.rank == r["rank"], (w.name, arm, rec.rank, r["rank"])
            assert rec.reach.L_anchor == r["L_anchor"], (w.name, arm)
            assert abs(rec.reach.J_old - r["J_old"]) <= 1e-5 * max(r["J_old"], 1.0), (w.name, arm)
            assert abs(rec.reach.A0q - ref["A0999"]) <= 1e-12 * max(abs(ref["A0999"]), 1.0)
            assert rec.sigma_max == pytest.approx(r["sigma_max"], rel=1e-9)
        op.close()
        n_checked += 1
    assert n_checked >= 1
