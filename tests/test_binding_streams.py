"""Stream selection of the Python binding (host logic, no GPU).

A device call on torch tensors with no stream must run on torch's current stream,
so that it is ordered after the torch work that produced its inputs; torch's
default stream has handle 0, which the C ABI reads as "the handle's own stream",
so the binding passes the CUDA runtime's explicit legacy-stream handle instead.
"""
import types

import pytest

from paper_2605_26580_gb300 import jbp


class _FakeCudaTensor:
    is_cuda = True
    device = "cuda:0"


def _patch_current_stream(monkeypatch, handle):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: types.SimpleNamespace(cuda_stream=handle))


def test_explicit_stream_passes_through(monkeypatch):
    _patch_current_stream(monkeypatch, 0)
    assert jbp._stream_ptr(types.SimpleNamespace(cuda_stream=1234), _FakeCudaTensor()) == 1234
    assert jbp._stream_ptr(5678, _FakeCudaTensor()) == 5678


def test_torch_default_stream_becomes_the_legacy_handle(monkeypatch):
    _patch_current_stream(monkeypatch, 0)
    assert jbp._stream_ptr(None, _FakeCudaTensor()) == jbp.CUDA_STREAM_LEGACY == 0x1


def test_torch_side_stream_is_used(monkeypatch):
    _patch_current_stream(monkeypatch, 0xABC0)
    assert jbp._stream_ptr(None, _FakeCudaTensor()) == 0xABC0


def test_host_buffers_use_the_handle_stream():
    assert jbp._stream_ptr(None, None) is None
    assert jbp._stream_ptr(None, types.SimpleNamespace(is_cuda=False)) is None
