"""The paper's interface (Sec. 3): model = BSC_ET(D, H, Hprime, gamma),
LinearAnnealing, standard_init, EM.run, inference -> res["s"], res["p"];
checkpoint/resume of the parameters."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from paper_1908_06843_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _recovered(Wl, Wtrue):
    a = Wl - Wl.mean(1, keepdims=True)
    b = Wtrue - Wtrue.mean(1, keepdims=True)
    C = (b / np.linalg.norm(b, axis=1, keepdims=True)) @ (a / np.linalg.norm(a, axis=1, keepdims=True)).T
    r, c = linear_sum_assignment(-C)
    return bool(np.all(C[r, c] > 0.95))


def test_bsc_em_run_and_inference():
    from paper_1908_06843_gb300 import BSC_ET, EM, LinearAnnealing
    d = synth.bars(N=1000, seed=1001)
    model = BSC_ET(25, 10, 6, 3)
    anneal = LinearAnnealing(50)
    p0 = synth.init_bsc(d["Y"], 10, seed=2001, pi=0.5, normalise=False)
    params = model._pack(p0["Wt"], p0["pi"], p0["sigma"])
    em = EM(model=model, anneal=anneal, data={"y": d["Y"]}, lparams=params)
    em.run()
    assert len(em.history) == 50 and np.all(np.isfinite(em.history))
    assert _recovered(em.lparams["W"].cpu().numpy(), d["Wt"])
    res = model.inference(anneal, em.lparams, d["Y"])
    s = res["s"].cpu().numpy()
    mi = res["map_idx"].cpu().numpy()
    for n in range(0, 1000, 37):
        assert set(np.flatnonzero(s[n])) == set(mi[n][mi[n] >= 0])
    p = res["p"].cpu().numpy()
    assert np.all((p > 0) & (p <= 1))


def test_checkpoint_resume():
    from paper_1908_06843_gb300 import BSC_ET, EM, LinearAnnealing, load_params, save_params
    import tempfile, os
    d = synth.bars(N=1000, seed=1001)
    p0 = synth.init_bsc(d["Y"], 10, seed=2001, pi=0.5, normalise=False)
    m1 = BSC_ET(25, 10, 6, 3)
    run20 = EM(m1, LinearAnnealing(20), {"y": d["Y"]}, m1._pack(p0["Wt"], p0["pi"], p0["sigma"])).run()
    m2 = BSC_ET(25, 10, 6, 3)
    half = EM(m2, LinearAnnealing(10), {"y": d["Y"]}, m2._pack(p0["Wt"], p0["pi"], p0["sigma"])).run()
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "ckpt.npz")
        save_params(f, half)
        resumed = load_params(f)
    run10 = EM(m2, LinearAnnealing(10), {"y": d["Y"]}, resumed).run()
    a, b = run20["W"].cpu().numpy(), run10["W"].cpu().numpy()
    # FP64 atomics sum in a run-dependent order: equal up to that rounding
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    assert abs(float(run20["theta"][1]) - float(run10["theta"][1])) <= 1e-6


def test_mca_and_gsc_models_run():
    from paper_1908_06843_gb300 import EM, GSC_ET, MCA_ET, LinearAnnealing
    d = synth.mca_bars(N=2000, seed=1003)
    m = MCA_ET(100, 20, 8, 4, rho=20.0)
    em = EM(m, LinearAnnealing(5), {"y": d["Y"]})
    em.run()
    assert np.all(np.isfinite(em.history))
    g = synth.gsc(N=2000, seed=1004)
    mg = GSC_ET(64, 32, 8, 3)
    emg = EM(mg, LinearAnnealing(5), {"y": g["Y"]})
    emg.run()
    assert np.all(np.isfinite(emg.history))
    assert emg.history[-1] > emg.history[0]
