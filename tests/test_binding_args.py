"""The Python binding's argument checks (host logic, no GPU): every tensor
whose pointer reaches librtt is checked for dtype, shape, contiguity, device
and agreement with the input, and a bad one raises ValueError before any
library call.  The library is replaced by a recorder and GPU residency is
faked, so the valid paths run through to the call on CPU tensors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2609_05528_b300 import rtt  # noqa: E402

S, K, T, R, RL = 6, 5, 4, 3, 2  # nodes, hats, frames, arm rows, mixed rows


class _Recorder:
    """Stands in for librtt: every entry point returns RTT_OK and is logged."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append(name)
            return 0
        return fn


@pytest.fixture
def fake(monkeypatch):
    rec = _Recorder()
    monkeypatch.setattr(rtt, "lib", lambda: rec)
    monkeypatch.setattr(rtt, "_on_gpu", lambda t: True)
    op = rtt.Operator.__new__(rtt.Operator)
    op.handle = None
    op.n_nodes, op.n_hats, op.n_frames = S, K, T
    op.arm_rows = lambda arm_mask=7: R if arm_mask == 7 else 1
    op.mix_rows_count = lambda mode, arm_mask=7: RL
    return op, rec


def f32(*shape):
    return torch.zeros(shape, dtype=torch.float32)


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def test_valid_calls_reach_the_library(fake):
    op, rec = fake
    assert op.apply_A(f32(S, K, 2), stream=0).shape == (R, T, 2)
    assert op.apply_A(f64(S, K, 3), y=f64(R, T, 3), stream=0).shape == (R, T, 3)
    assert op.apply_A(f32(S, K, 2), arm_mask=1, stream=0).shape == (1, T, 2)
    assert op.apply_AT(f32(R, T, 2), stream=0).shape == (S, K, 2)
    assert op.apply_AT(f64(1, T, 2), x=f64(S, K, 2), arm_mask=1, stream=0).shape == (S, K, 2)
    y, g = op.apply_A_AT(f32(S, K, 4), d=f32(R, T, 4), stream=0)
    assert y.shape == (R, T, 4) and g.shape == (S, K, 4)
    assert op.mix_rows(f32(R, T, 2), rtt.MIX_UNRESOLVED, stream=0).shape == (RL, T, 2)
    assert op.mix_rows_T(f64(RL, T, 2), rtt.MIX_TOTAL_FLUX, stream=0).shape == (R, T, 2)
    assert rtt.gram(op, f64(S, K, 7), stream=0).shape == (7, 7)
    assert rtt.gram_normal_mix(op, f64(S, K, 7), rtt.MIX_UNRESOLVED, stream=0).shape == (7, 7)
    ev, V, _ = rtt.eig_sym(f64(4, 4), stream=0)
    assert ev.shape == (4,) and V.shape == (4, 4)
    assert rtt.eigvals_sym_batched(f64(3, 4, 4), stream=0).shape == (3, 4)
    x, _, rel = rtt.solve_ridge(op, f32(R, T, 2), [0.1, 1.0], stream=0)
    assert x.shape == (S, K, 4) and rel.shape == (4,)
    xh = rtt.solve_tsvd(op, f64(S, K, 3), f64(3, 3), np.ones(3), 2, f64(R, T, 2), stream=0)
    assert xh.shape == (S, K, 2)
    for name in ("rtt_apply_A", "rtt_apply_A_f64", "rtt_apply_AT", "rtt_apply_AT_f64",
                 "rtt_apply_A_AT", "rtt_mix_rows", "rtt_mix_rows_T_f64", "rtt_gram",
                 "rtt_gram_normal_mix", "rtt_eig_sym", "rtt_eigvals_sym_batched",
                 "rtt_solve_ridge", "rtt_solve_tsvd"):
        assert name in rec.calls, name


@pytest.mark.parametrize("call, msg", [
    (lambda op: op.apply_A(f32(S, K + 1, 2), stream=0), "shape"),
    (lambda op: op.apply_A(f32(S, K), stream=0), "shape"),
    (lambda op: op.apply_A(torch.zeros((S, K, 2), dtype=torch.int32), stream=0), "dtype"),
    (lambda op: op.apply_A(f32(S, 2, K).transpose(1, 2), stream=0), "contiguous"),
    (lambda op: op.apply_A(np.zeros((S, K, 2), np.float32), stream=0), "torch tensor"),
    (lambda op: op.apply_A(f32(S, K, 2), y=f32(R + 1, T, 2), stream=0), "shape"),
    (lambda op: op.apply_A(f32(S, K, 2), y=f32(R, T, 3), stream=0), "shape"),
    (lambda op: op.apply_A(f32(S, K, 2), y=f64(R, T, 2), stream=0), "dtype"),
    (lambda op: op.apply_A(f32(S, K, 2), y=f32(1, T, 2), arm_mask=7, stream=0), "shape"),
    (lambda op: op.apply_AT(f32(R, T, 2), arm_mask=1, stream=0), "shape"),
    (lambda op: op.apply_AT(f32(R, T + 1, 2), stream=0), "shape"),
    (lambda op: op.apply_AT(f32(R, T, 2), x=f32(S, K, 3), stream=0), "shape"),
    (lambda op: op.apply_A_AT(f64(S, K, 2), stream=0), "dtype"),
    (lambda op: op.apply_A_AT(f32(S, K, 2), d=f32(R, T, 3), stream=0), "shape"),
    (lambda op: op.apply_A_AT(f32(S, K, 2), g=f32(S, K, 1), stream=0), "shape"),
    (lambda op: op.apply_A_AT(f32(S, K, 2), y=f32(R, 2, T).transpose(1, 2), stream=0),
     "contiguous"),
    (lambda op: op.mix_rows(f32(RL, T, 2), rtt.MIX_UNRESOLVED, stream=0), "shape"),
    (lambda op: op.mix_rows(f32(R, T, 2), rtt.MIX_UNRESOLVED, out=f32(R, T, 2), stream=0), "shape"),
    (lambda op: op.mix_rows_T(f32(R, T, 2), rtt.MIX_UNRESOLVED, stream=0), "shape"),
    (lambda op: op.mix_rows_T(f32(RL, T, 2), rtt.MIX_UNRESOLVED, out=f64(R, T, 2), stream=0),
     "dtype"),
    (lambda op: rtt.gram(op, f32(S, K, 7), stream=0), "dtype"),
    (lambda op: rtt.gram(op, f64(S + 1, K, 7), stream=0), "shape"),
    (lambda op: rtt.gram_normal_mix(op, f64(S, K), rtt.MIX_TOTAL_FLUX, stream=0), "shape"),
    (lambda op: rtt.eig_sym(f64(4, 5), stream=0), "shape"),
    (lambda op: rtt.eig_sym(f32(4, 4), stream=0), "dtype"),
    (lambda op: rtt.eigvals_sym_batched(f64(4, 4), stream=0), "shape"),
    (lambda op: rtt.solve_ridge(op, f64(R, T, 2), [1.0], stream=0), "dtype"),
    (lambda op: rtt.solve_ridge(op, f32(R, T, 2), [1.0], arm_mask=1, stream=0), "shape"),
    (lambda op: rtt.solve_tsvd(op, f64(S, K, 3), f64(3, 2), np.ones(3), 2, f64(R, T, 2),
                               stream=0), "shape"),
    (lambda op: rtt.solve_tsvd(op, f64(S, K, 3), f64(3, 3), np.ones(2), 2, f64(R, T, 2),
                               stream=0), "evals"),
    (lambda op: rtt.solve_tsvd(op, f64(S, K, 3), f64(3, 3), np.ones(3), 2, f32(R, T, 2),
                               stream=0), "dtype"),
    (lambda op: rtt.rank_audit([op], [f64(S, K, 5), None], stream=0), "entries"),
    (lambda op: rtt.rank_audit([op, op], [f64(S, K, 5), f64(S, K, 6)], stream=0), "shape"),
])
def test_bad_arguments_raise_before_the_library(fake, call, msg):
    op, rec = fake
    with pytest.raises(ValueError, match=msg):
        call(op)
    assert rec.calls == []


def test_host_tensors_are_refused(monkeypatch):
    """Without the fake residency, a correctly shaped host tensor is refused."""
    rec = _Recorder()
    monkeypatch.setattr(rtt, "lib", lambda: rec)
    op = rtt.Operator.__new__(rtt.Operator)
    op.handle = None
    op.n_nodes, op.n_hats, op.n_frames = S, K, T
    op.arm_rows = lambda arm_mask=7: R
    with pytest.raises(ValueError, match="CUDA"):
        op.apply_A(f32(S, K, 2), stream=0)
    with pytest.raises(ValueError, match="CUDA"):
        rtt.gram(op, f64(S, K, 3), stream=0)
    assert rec.calls == []


def test_missing_library_fails_loudly(monkeypatch):
    """Without librtt.so every entry point raises: there is no CPU fallback."""
    monkeypatch.setattr(rtt, "_LIB", None)
    monkeypatch.setattr(rtt, "LIB_PATH", "/nonexistent/librtt.so")
    with pytest.raises(RuntimeError, match="missing"):
        rtt.lib()
    with pytest.raises(RuntimeError, match="missing"):
        rtt.class_dim(rtt.CLASS_S224)
