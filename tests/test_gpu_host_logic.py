"""Host-side library behaviour on the GPU: concurrent host threads, the plan cache's eviction,
explicit plans on several streams, and CUDA-graph capture of the plan entry points."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import inputs  # noqa: E402
from oracle import radial as oradial  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_concurrent_host_threads_with_different_mode_lists():
    r = inputs.uniform_points(300, 5)[0]
    rt = torch.as_tensor(r, device=DEV)
    jobs = [inputs.radial_modes(n) for n in (4, 9, 15, 22)]
    want = [np.array(oradial.radial_table(ns, ms, r, 1)) for ns, ms in jobs]
    results, errors = {}, []

    def work(i):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(5):
                    out = zp.radial(jobs[i][0], jobs[i][1], rt, 1)
                s.synchronize()
                results[i] = out.cpu().numpy()
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(jobs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, w in enumerate(want):
        assert np.max(np.abs(results[i] - w)) < 1e-9


def test_plan_cache_eviction_keeps_results_correct():
    """More distinct mode lists than the cache holds (64): every call still matches."""
    r = inputs.uniform_points(64, 6)[0]
    rt = torch.as_tensor(r, device=DEV)
    for k in range(70):
        ns = [k, k + 2]
        ms = [k % 2, k % 2]
        out = zp.radial(ns, ms, rt, 0).cpu().numpy()
        if k % 17 == 0:
            want = np.array(oradial.radial_table(ns, ms, r, 0))
            assert np.max(np.abs(out - want)) < 1e-12


@pytest.mark.parametrize("P", [1000, 10000])
def test_plan_entry_points_capture_in_a_cuda_graph(P):
    """1000 points: the walk alone; 10000 points: the point-table kernel and its stream-ordered
    scratch allocation are captured too."""
    ns, ms = inputs.full_zernike_modes(12)
    r, th = inputs.uniform_points(P, 7)
    rt, tt = torch.as_tensor(r, device=DEV), torch.as_tensor(th, device=DEV)
    plan = zp.Plan(ns, ms)
    ref, _ = zp.basis(None, None, rt, tt, 2, plan=plan)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            out, _ = zp.basis(None, None, rt, tt, 2, plan=plan)
    torch.cuda.current_stream().wait_stream(s)
    rt.add_(0.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # new inputs in the same buffers, replay again
    r2 = inputs.uniform_points(P, 8)[0]
    rt.copy_(torch.as_tensor(r2, device=DEV))
    g.replay()
    torch.cuda.synchronize()
    ref2, _ = zp.basis(None, None, rt, tt, 2, plan=plan)
    assert torch.equal(out, ref2)


def test_release_scratch_returns_ok_and_calls_keep_working():
    """zp_release_scratch trims the library's scratch pool after a synchronisation; a call that
    needs scratch afterwards allocates again and gives the same result."""
    import numpy as np
    import paper_2409_19156_gb300 as zp
    from paper_2409_19156_gb300 import _lib, inputs

    ns, ms = inputs.full_zernike_modes(12)
    r, th = inputs.uniform_points(3000, 3)
    C = np.random.default_rng(3).standard_normal((len(ns), 8))
    rt, tt, Ct = (torch.as_tensor(x, device="cuda:0") for x in (r, th, C))
    before = zp.series_eval(ns, ms, rt, tt, Ct, "fp64emu")
    torch.cuda.synchronize()
    lib = _lib.load()
    assert lib.zp_release_scratch() == 0
    after = zp.series_eval(ns, ms, rt, tt, Ct, "fp64emu")
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    assert lib.zp_release_scratch() == 0


def test_tuner_cache_persists_across_calls(tmp_path, monkeypatch):
    """zp_batch_tune keeps its result per GPU and batch shape: with ZP_TUNE_CACHE naming a file,
    the key and configuration are written there, and a second tune of the same batch returns
    the stored configuration without timing again."""
    import time

    path = tmp_path / "tune.txt"
    monkeypatch.setenv("ZP_TUNE_CACHE", str(path))
    rng = np.random.default_rng(4)
    inst = []
    for k, (n_max, P) in enumerate([(6, 300), (11, 257), (3, 40)]):
        ns, ms = inputs.full_zernike_modes(n_max)
        r, th = inputs.uniform_points(P, 40 + k)
        inst.append({"n": ns, "m": ms, "r": torch.as_tensor(r, device=DEV), "theta": torch.as_tensor(th, device=DEV),
                     "coeffs": torch.as_tensor(rng.standard_normal((len(ns), 5)), device=DEV)})
    b = zp.Batch(inst, 5, with_adjoint=False)
    cfg1, ms1 = b.tune("forward", "fp64", reps=1)
    text = path.read_text()
    assert "/inst3/" in text and "/sets5/" in text
    t0 = time.perf_counter()
    cfg2, ms2 = b.tune("forward", "fp64", reps=1)
    assert time.perf_counter() - t0 < 0.05  # no candidate launched
    assert cfg2 == cfg1 and ms2 == ms1
    assert b.config() == cfg1


def test_debug_level_checks_and_logs_every_call(tmp_path):
    """ZP_DEBUG=2: every compute entry point synchronises, checks and logs one line."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import torch, paper_2409_19156_gb300 as zp\n"
            "r = torch.linspace(0, 1, 64, dtype=torch.float64, device='cuda:0')\n"
            "zp.radial([2, 3], [0, 1], r, 1)\n"
            "zp.series_eval([2, 3], [0, 1], r, r, torch.ones(2, 3, dtype=torch.float64, device='cuda:0'))\n"
            "torch.cuda.synchronize()\n")
    env = dict(os.environ, ZP_DEBUG="2", PYTHONPATH=root)
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    assert "[zp] zp_radial -> 0" in res.stderr
    assert "[zp] zp_series_eval -> 0" in res.stderr
