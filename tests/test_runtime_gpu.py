"""Runtime services around the C ABI, on the GPU: the bounds-checked build
(the stand-in for a memory sanitizer) running small-N parity cases, per-call
JSON-lines metrics, and the persistent autotuner cache with the LM_AUTOTUNE
switch.  Each case runs in a child process so that the environment switch
and the library it selects apply from the first load."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2510_02135_gb300 import _build

    _build.build()


def _child(code, env_extra, timeout=600):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=timeout)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


_PARITY_CASES = r'''
import sys
sys.path.insert(0, ".")
sys.path.insert(0, "tests")
import numpy as np, torch
import oracle
from paper_2510_02135_gb300 import inputs as I, lm
assert lm.lm_debug_bounds(), "not the bounds-checked library"
oracle.build()
dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
def rel(y, r):
    y = np.asarray(y, np.float64).ravel(); r = np.asarray(r, np.float64).ravel()
    return float(np.linalg.norm(y - r) / max(np.linalg.norm(r), 1e-300))
worst = 0.0
for n in (1, 2, 3, 31, 33, 129, 700):
    for fp64 in (False, True):
        s_ = I.cube_suspension(100 + n, n, 0.15, 1.0, angular=True, fp32=not fp64)
        ur, wr = oracle.mdot(s_.pos, s_.F, s_.T, 1.0, 1.0, True)
        s = lm.lm_create(1.0, 1.0, True, lm.LM_FP64 if fp64 else lm.LM_FP32C)
        lm.lm_set_positions(s, dev(s_.pos))
        cfgs = [(128, 1, 1, 0), (256, 2, 3, 0)] if fp64 else [(128, 2, 1, 2), (256, 8, 5, 2), (128, 4, 2, 0)]
        for cfg in cfgs:
            lm.lm_set_pair_config(s, *cfg)
            u, w = lm.lm_mdot(s, dev(s_.F), dev(s_.T))
            e = max(rel(u.cpu(), ur), rel(w.cpu(), wr))
            assert e < (1e-12 if fp64 else 1e-5), (n, fp64, cfg, e)
            worst = max(worst, e)
        if n >= 31:
            lin, ang, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=1e-6, max_iter=6 * n)
            y = np.concatenate([lin.cpu().numpy().ravel(), ang.cpu().numpy().ravel()])
            ex = oracle.sqrt_exact(oracle.assemble(s_.pos, 1.0, 1.0, True), s_.W)
            assert rel(y, ex) < 2e-5, (n, fp64, rel(y, ex))
    # adjoint (translation, packed) and the single-wall product
    s_ = I.cube_suspension(200 + n, n, 0.15, 1.0, angular=False, fp32=True)
    s = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C)
    lm.lm_set_positions(s, dev(s_.pos))
    dX, dF, _ = lm.lm_mdot_backward(s, dev(s_.F), None, dev(s_.G), None)
    g = oracle.grad(s_.pos, s_.F, None, s_.G, None, 1.0, 1.0, False)
    if n > 1:
        assert rel(dX.cpu(), g) < 1e-4, (n, rel(dX.cpu(), g))
    lm.lm_set_adjoint_config(s, 128, 2, 0, 3)   # the symmetric form
    dX, dF, _ = lm.lm_mdot_backward(s, dev(s_.F), None, dev(s_.G), None)
    if n > 1:
        assert rel(dX.cpu(), g) < 1e-4, (n, "symmetric", rel(dX.cpu(), g))
    # the symmetric adjoint with angular blocks: FP32 scalar (ilp 2, 4), FP32 packed, FP64
    for fp64, ilp, packed in ((False, 2, 3), (False, 4, 3), (False, 2, 4), (False, 4, 4), (True, 1, 3)):
        sa = I.cube_suspension(300 + n, n, 0.15, 1.0, angular=True, fp32=not fp64)
        s = lm.lm_create(1.0, 1.0, True, lm.LM_FP64 if fp64 else lm.LM_FP32C)
        lm.lm_set_positions(s, dev(sa.pos))
        lm.lm_set_adjoint_config(s, 128, ilp, 0, packed)
        dX, dF, dT = lm.lm_mdot_backward(s, dev(sa.F), dev(sa.T), dev(sa.G), dev(sa.H))
        g = oracle.grad(sa.pos, sa.F, sa.T, sa.G, sa.H, 1.0, 1.0, True)
        gt = oracle.mdot(sa.pos, sa.G, sa.H, 1.0, 1.0, True)[1]
        if n > 1:
            assert rel(dX.cpu(), g) < 1e-4, (n, fp64, ilp, packed, "symmetric 6N", rel(dX.cpu(), g))
        assert rel(dT.cpu(), gt) < 1e-4, (n, fp64, ilp, packed, "symmetric 6N dT", rel(dT.cpu(), gt))
    pw = s_.pos.copy(); pw[:, 2] -= pw[:, 2].min() - 0.5
    sw = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C, periodicity=("open", "open", "single_wall"))
    lm.lm_set_positions(sw, dev(pw))
    uw, _ = lm.lm_mdot(sw, dev(s_.F), None)
    uwr, _ = oracle.mdot(pw, s_.F, None, 1.0, 1.0, False, wall=True)
    assert rel(uw.cpu(), uwr) < 1e-5
# a small batch: one Brownian step
b_ = I.batch_suspensions(7, S=5, nmin=20, nmax=300)
b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
lm.lm_batch_set_positions(b, dev(b_.pos))
lm.lm_batch_bd_run(b, 1.0, 1e-3, 1.0, 2, step0=0, seed=3, tol=1e-4, use_graph=False)
# the device tridiagonal step: the warp quadrature and its QR fallback (graded T)
rng = np.random.default_rng(4)
for m in (1, 7, 40, 128):
    al = rng.uniform(0.5, 3.0, (3, m)); be = rng.uniform(0.05, 0.8, (3, m))
    al[0] = rng.uniform(2.0, 3.0, m); be[0] = rng.uniform(0.05, 0.5, m)   # diagonally dominant: certified
    al[2] = np.linspace(1e-7, 1.0, m); be[2] = 1e-9                          # graded: the QR form
    out, paths = lm.lm_tridiag_sqrt_e1_device(torch.from_numpy(al).cuda(), torch.from_numpy(be).cuda(), paths=True)
    for c in range(3):
        want = oracle.tridiag_sqrt_e1(al[c], be[c, : m - 1])
        got = out[c].cpu().numpy()
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), (m, c)
    assert paths[0] == 0 and (m == 1 or paths[2] == 1), (m, list(paths))
torch.cuda.synchronize()
lm.lm_debug_check()
print("bounds-checked parity ok, worst M[F;T] error %.2e" % worst)
'''


def test_bounds_checked_build_runs_small_cases_clean():
    """The bounds-checked library (-DLM_DEBUG_BOUNDS) on N = 1, 2, 3, 31, 33,
    129, 700 (non-multiples of every tile size), FP32 and FP64, packed and
    scalar tilings, one and several j-splits, the Lanczos root, the adjoint,
    the single wall and a small batch: every result matches the oracle and no
    device index check fails (lm_debug_check)."""
    from paper_2510_02135_gb300 import _build

    _build.build(debug_bounds=True)
    out = _child(_PARITY_CASES, {"LM_DEBUG_BOUNDS": "1"}, timeout=900)
    assert "bounds-checked parity ok" in out


def test_release_build_reports_no_bounds_checks():
    from paper_2510_02135_gb300 import lm

    if os.environ.get("LM_DEBUG_BOUNDS") == "1":
        pytest.skip("the bounds-checked build is loaded")
    assert not lm.lm_debug_bounds()
    lm.lm_debug_check()


def test_metrics_jsonl_one_line_per_call(tmp_path):
    path = tmp_path / "calls.jsonl"
    code = r'''
import sys; sys.path.insert(0, ".")
import numpy as np, torch
from paper_2510_02135_gb300 import inputs as I, lm
s_ = I.cube_suspension(5, 2000, 0.1, 1.0, angular=True, fp32=True)
dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
s = lm.lm_create(1.0, 1.0, True, lm.LM_FP32C)
lm.lm_set_positions(s, dev(s_.pos))
lm.lm_mdot(s, dev(s_.F), dev(s_.T))
lin, ang, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=1e-5)
print(it)
'''
    out = _child(code, {"LM_METRICS_JSONL": str(path)})
    its = int(out.strip().splitlines()[-1])
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    calls = [x["call"] for x in lines]
    assert calls == ["lm_mdot", "lm_sqrt_mdot"], calls
    m, q = lines
    assert m["status"] == 0 and m["N"] == 2000 and m["angular"] == 1 and m["precision"] == "fp32c"
    assert m["pair_interactions"] == 2000.0 ** 2 and m["flops_per_pair"] == 86 and m["ms"] > 0
    assert q["iterations"] == its and q["converged"] == 1 and q["products"] == its
    assert q["rel_change"] < 1e-5 and q["sms"] > 0 and q["fp32_peak_tflops"] > 0 and q["gpu"]


def test_autotune_cache_persists_across_processes(tmp_path):
    """lm_autotune's choice lands in LM_AUTOTUNE_CACHE and a fresh process
    starts from it; with LM_AUTOTUNE=1 a solver tunes on first use by itself."""
    cache = tmp_path / "tune.jsonl"
    tune = r'''
import sys; sys.path.insert(0, ".")
import numpy as np, torch
from paper_2510_02135_gb300 import inputs as I, lm
s_ = I.cube_suspension(6, 3000, 0.1, 1.0, angular=False, fp32=True)
s = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C)
lm.lm_set_positions(s, torch.from_numpy(s_.pos).cuda())
MODE
print(lm.lm_get_pair_config(s))
'''
    out1 = _child(tune.replace("MODE", "lm.lm_autotune(s, reps=1)"), {"LM_AUTOTUNE_CACHE": str(cache)})
    entries = [json.loads(x) for x in cache.read_text().splitlines()]
    assert len(entries) == 1 and entries[0]["n"] == 3000 and entries[0]["angular"] == 0
    out2 = _child(tune.replace("MODE", "pass"), {"LM_AUTOTUNE_CACHE": str(cache)})
    assert out1.strip().splitlines()[-1] == out2.strip().splitlines()[-1]
    cache2 = tmp_path / "tune2.jsonl"
    _child(tune.replace("MODE", "lm.lm_mdot(s, torch.from_numpy(s_.F).cuda(), None)"),
           {"LM_AUTOTUNE_CACHE": str(cache2), "LM_AUTOTUNE": "1"})
    assert len(cache2.read_text().splitlines()) == 1
