"""GPU: the learned surrogate end to end -- data from the batched complex64
march (checked against the FP64 oracle), an ensemble of four networks
trained by the library's own tensor-core kernels, calibration of its error
estimate on solver runs it never saw, and what it gains over the march alone
on held-out parameters, with the march as the fallback.

Sizes: 20480 training runs, 1024 calibration runs and 512 held-out runs of
the surrogate grid (1024 x 1024, delta = 0.05), four networks 4 -> 512 x 4 ->
512 trained for 60000 Adam steps of 512 samples each (about a minute in all).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05943_gb300 import build, surrogate as S
    build.build()
    return torch, S


@pytest.fixture(scope="module")
def data(env):
    torch, S = env
    wtr, ftr = W.surrogate_draw(17070, 20480)
    wca, fca = W.surrogate_draw(17072, 1024)
    wte, fte = W.surrogate_draw(17071, 512)
    Ytr, ttr = S.march_targets(wtr)
    Yca, _ = S.march_targets(wca)
    Yte, tte = S.march_targets(wte)
    print(f"march data: {len(wtr)} runs in {ttr:.1f} s; held-out {len(wte)} runs in {tte:.2f} s")
    return dict(wtr=wtr, ftr=ftr, Ytr=Ytr, fca=fca, Yca=Yca, wte=wte, fte=fte, Yte=Yte, tte=tte)


@pytest.fixture(scope="module")
def trained(env, data):
    torch, S = env
    sur = S.Surrogate(K=4, outputs="norm", ranges=W.SURR_RANGES)
    log = sur.fit(S.normalise(data["ftr"], W.SURR_RANGES), data["Ytr"], steps=60000, batch=512, lr=2e-3)
    print(f"training: {log.steps} steps x 4 networks in {log.seconds:.1f} s, final losses {log.final_loss}")
    q = sur.calibrate(S.normalise(data["fca"], W.SURR_RANGES), data["Yca"])
    print(f"calibration factor of the ensemble spread: {q:.3f}")
    return sur


def test_training_data_matches_oracle(env, data, oracle):
    # the targets of two held-out runs, recomputed from the FP64 oracle's march
    torch, S = env
    for i in (0, 1):
        w = data["wte"][i]
        p = oracle.Params(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                          init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center)
        r = oracle.march(p, tstep=15)
        want = S.targets_from_march(r["norms"], r["snaps"], w)
        assert np.max(np.abs(want - data["Yte"][i])) <= 1e-6 * max(1.0, np.max(np.abs(want)))


def test_held_out_error(env, data, trained):
    torch, S = env
    mean, est = trained.predict(S.normalise(data["fte"], W.SURR_RANGES))
    err = np.abs(mean - data["Yte"][:, trained.cols]).max(axis=1)
    print(f"held-out max |N - N_march| per run: median {np.median(err):.2e}, 90th pct "
          f"{np.percentile(err, 90):.2e}, worst {err.max():.2e}; within {TOL:g}: {np.mean(err <= TOL):.1%}")
    assert np.median(err) < 2 * TOL
    # the spread ranks the errors: the runs it flags worst hold the largest errors
    assert np.corrcoef(np.log(est), np.log(err))[0, 1] > 0.5


def test_fallback_and_gain(env, data, trained):
    torch, S = env
    wte, fte, Yte = data["wte"], data["fte"], data["Yte"]
    out, served, t_net, t_march = trained.answer(wte, fte, tol=TOL)
    err = np.abs(out - Yte[:, trained.cols]).max(axis=1)
    # queries the network answers are within the tolerance (calibrated at the 99th percentile)
    assert served.mean() > 0.05
    assert np.mean(err[served] <= TOL) >= 0.98 and err[served].max() <= 2 * TOL
    # queries it declines are the march's own answer
    assert np.all(err[~served] <= 1e-6)
    per_query_net = t_net / len(wte)
    per_query_march = data["tte"] / len(wte)
    total = t_net + t_march
    print(f"served by the network: {served.mean():.1%} (worst error {err[served].max():.2e}); "
          f"per query: network {per_query_net * 1e3:.3f} ms vs march {per_query_march * 1e3:.3f} ms; "
          f"all {len(wte)} queries: {total:.3f} s with the network vs {data['tte']:.3f} s march alone "
          f"({data['tte'] / total:.2f}x)")
    assert per_query_march > 10 * per_query_net
