"""CPU: the autotuner's host logic with a stand-in timer -- it measures every
candidate once, keeps the fastest, keys the cache by batch shape and answers
from the cache afterwards (no GPU work)."""
import workloads as W
from paper_1707_05943_gb300 import autotune as A
from paper_1707_05943_gb300 import fdtd as F


def cfgs(ws):
    return [F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                     init_cond=w.init_cond, sigma=w.sigma, center=w.center, precision=F.F32_COMP) for w in ws]


def test_tune_picks_fastest_and_caches(tmp_path):
    c = cfgs(W.batch(n=16, nx_hi=1 << 12))
    calls = []

    def timer(configs, cl, w, rows):
        calls.append((cl, w))
        return 10.0 + abs(cl - 16) + abs(w - 32) / 8.0  # fastest at (16, 32)

    path = str(tmp_path / "cache.json")
    ch = A.tune(c, rows=64, cache_path=path, timer=timer)
    assert (ch.cluster_ctas, ch.mid_weight) == (16, 32)
    assert sorted(calls) == sorted(A.CANDIDATES) and len(ch.table) == len(A.CANDIDATES)
    calls.clear()
    again = A.tune(c, rows=64, cache_path=path, timer=timer)
    assert calls == [] and (again.cluster_ctas, again.mid_weight) == (16, 32) and again.key == ch.key
    A.tune(c, rows=64, cache_path=path, timer=timer, refresh=True)
    assert len(calls) == len(A.CANDIDATES)


def test_bucket_separates_shapes():
    a = A.bucket(cfgs(W.batch(n=16, nx_hi=1 << 12)))
    b = A.bucket(cfgs(W.batch(n=64, nx_hi=1 << 12)))
    c = A.bucket(cfgs(W.batch(n=16, nx_lo=1 << 14, nx_hi=1 << 16)))
    assert len({a, b, c}) == 3
    assert a == A.bucket(cfgs(W.batch(n=16, nx_hi=1 << 12)))
