"""Autotuner logic on the CPU (timings injected), and on the GPU (real timings)."""
import pytest


def test_bucket_and_choice(tmp_path):
    from paper_2511_01255_gb300 import autotune as A
    assert A.n_bucket(1000) == A.n_bucket(1010) != A.n_bucket(1400)
    assert A.choose({32: 2.0, 64: 1.0, 128: 1.0}) == 64


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_2511_01255_gb300 import autotune as A
    calls = []

    def fake(N, k1, k2, NP, team, comp, form, gens):
        calls.append(team)
        return {32: 3.0, 64: 2.0, 128: 1.5, 256: 1.7}[team]

    import types
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        is_available=lambda: False, get_device_name=lambda: "cpu"))
    monkeypatch.setitem(__import__("sys").modules, "torch", fake_torch)
    path = str(tmp_path / "cache.json")
    t = A.autotune_team(1000, 1.0, 2.0, 256, form=2, measure=fake, path=path)
    assert t == 128 and sorted(calls) == [32, 64, 128, 256]
    calls.clear()
    assert A.autotune_team(1000, 1.0, 2.0, 256, form=2, measure=fake, path=path) == 128
    assert calls == []  # served from the cache


@pytest.mark.gpu
def test_autotune_on_gpu(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    from paper_2511_01255_gb300 import autotune as A
    t = A.autotune_team(1000, 0.9, 4.0, 64, compensated=1, form=q.RUN_PERSISTENT, gens=10,
                        path=str(tmp_path / "c.json"))
    assert t in (32, 64, 128, 256)
