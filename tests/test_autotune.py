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


def test_objective_has_its_own_cache_entry(tmp_path, monkeypatch):
    """A multi-wavelength objective is tuned and cached apart from the single problem
    of the same size (its kernels differ), and per number of problems."""
    from paper_2511_01255_gb300 import autotune as A
    seen = []

    def fake(N, k1, k2, NP, team, comp, form, gens, objective=None):
        seen.append((team, objective is not None))
        base = {32: 3.0, 64: 1.0, 128: 1.5, 256: 2.0} if objective else {32: 3.0, 64: 2.0, 128: 1.0, 256: 1.2}
        return base[team]

    import types
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        is_available=lambda: False, get_device_name=lambda: "cpu"))
    monkeypatch.setitem(__import__("sys").modules, "torch", fake_torch)
    path = str(tmp_path / "cache.json")
    obj3 = (2, [(1.0, 2.0), (1.1, 2.1), (1.2, 2.2)], 1e5, 0.5)
    assert A.autotune_team(1000, 1.0, 2.0, 256, form=0, measure=fake, path=path) == 128
    assert A.autotune_team(1000, 1.0, 2.0, 256, form=0, measure=fake, path=path,
                           objective=obj3) == 64
    assert all(o for t, o in seen[4:]) and not any(o for t, o in seen[:4])
    n = len(seen)
    assert A.autotune_team(1000, 1.0, 2.0, 256, form=0, measure=fake, path=path,
                           objective=obj3) == 64
    assert len(seen) == n  # cached
    A.autotune_team(1000, 1.0, 2.0, 256, form=0, measure=fake, path=path,
                    objective=(2, obj3[1][:2], 1e5, 0.5))
    assert len(seen) == n + 4  # two problems: a new entry


@pytest.mark.gpu
def test_autotune_on_gpu(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    from paper_2511_01255_gb300 import autotune as A
    t = A.autotune_team(1000, 0.9, 4.0, 64, compensated=1, form=q.RUN_PERSISTENT, gens=10,
                        path=str(tmp_path / "c.json"))
    assert t in A.CANDIDATES
    obj = (3, [(2.1, 0.0), (2.4, 0.0), (2.9, 0.0)], 1.0e3, 0.5)
    t = A.autotune_team(1000, 2.1, 0.0, 64, form=q.RUN_LAUNCHES, gens=4,
                        path=str(tmp_path / "c.json"), objective=obj)
    assert t in A.CANDIDATES


def test_batch_cluster_choice_and_cache(tmp_path, monkeypatch):
    from paper_2511_01255_gb300 import autotune as A
    import types
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        is_available=lambda: False, get_device_name=lambda: "cpu"))
    monkeypatch.setitem(__import__("sys").modules, "torch", fake_torch)

    class FakeState:
        def __init__(self):
            self.problems = [(1000, 1.0, 2.0), (8000, 1.0, 2.0)]
            self.params = [types.SimpleNamespace(NP=64), types.SimpleNamespace(NP=512)]
            self.ctas = None

        def set_batch_cluster(self, c):
            self.ctas = c

    calls = []

    def fake(state, ctas, gens):
        calls.append(ctas)
        return {1: 5.0, 2: 4.5, 4: 4.7}[ctas]

    path = str(tmp_path / "cache.json")
    st = FakeState()
    assert A.autotune_batch_cluster(st, measure=fake, path=path) == 2 and st.ctas == 2
    assert sorted(calls) == [1, 2, 4]
    calls.clear()
    st2 = FakeState()
    assert A.autotune_batch_cluster(st2, measure=fake, path=path) == 2 and st2.ctas == 2
    assert calls == []  # served from the cache
    # another batch shape is another entry
    st3 = FakeState()
    st3.params[1].NP = 64
    A.autotune_batch_cluster(st3, measure=fake, path=path)
    assert sorted(calls) == [1, 2, 4]


@pytest.mark.gpu
def test_autotune_batch_cluster_on_gpu(tmp_path):
    """A real measurement on a small batch picks a valid size and leaves the state
    initialised with the same population as before."""
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    from paper_2511_01255_gb300 import autotune as A
    probs = [(300 + 100 * k, 0.9, 4.0) for k in range(6)]
    prms = [q.Params(16 + 8 * k, 200, 0.5, 0.9, 3, 0, 0) for k in range(6)]
    with q.State(probs, prms) as st:
        st.init()
        before = [st.population(k)[0].cpu().numpy() for k in range(6)]
        c = A.autotune_batch_cluster(st, gens=5, path=str(tmp_path / "c.json"))
        assert c in (1, 2, 4)
        assert st.generation == 0
        after = [st.population(k)[0].cpu().numpy() for k in range(6)]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        st.run(2, q.RUN_BATCHED)  # carries on with the chosen size
