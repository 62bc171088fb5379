"""bench.py on the host (no GPU): every global name its functions use is defined, the recorded
traffic tables are well formed, the algorithmic work per evaluation is the stated one, the
oracle arm (--impl reference) prints its one line on rank 0 only, with the GPU arm's workload config,
and the CPU context leg (the paper's FP32 Fourier variant) computes the oracle's log P."""
import builtins
import importlib
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def _global_names(code):
    names = set(code.co_names)
    for c in code.co_consts:
        if isinstance(c, types.CodeType):
            names |= _global_names(c)
    return names


def test_every_global_name_in_bench_is_defined():
    bench = _bench()
    missing = {}
    for name, obj in vars(bench).items():
        if isinstance(obj, types.FunctionType) and obj.__module__ == "bench":
            code = obj.__code__
            # co_names also holds attribute names; keep those loaded as globals
            import dis
            loads = set()

            def scan(c):
                for ins in dis.get_instructions(c):
                    if ins.opname in ("LOAD_GLOBAL", "LOAD_NAME"):
                        loads.add(ins.argval)
                for k in c.co_consts:
                    if isinstance(k, types.CodeType):
                        scan(k)
            scan(code)
            bad = {n for n in loads if not hasattr(bench, n) and not hasattr(builtins, n)}
            if bad:
                missing[name] = sorted(bad)
    assert not missing, missing


def test_kernel_identity_ignores_comments_only():
    """A stored DRAM figure stays attached to a kernel while only its comments change."""
    bench = _bench()
    code = "a = b; // note\n/* block\n comment */ c = d;   \n\n"
    assert bench._code_only(code) == bench._code_only("a = b;\n c = d;")
    assert bench._code_only(code) != bench._code_only("a = b;\n c = e;")


def test_traffic_tables_and_work_per_eval():
    bench = _bench()
    # a stored figure names the kernel source it was taken on ("" until one is taken)
    for k in ("k_score", "k_score_gemm", "k_score_tc"):
        assert len(bench.kernel_source_sha(k)) == 64
    assert len(bench.K_SCORE_TRAFFIC["source_sha256"]) == 64 and bench.K_SCORE_TRAFFIC["bytes_per_pair"] > 0
    t = bench.K_SCORE_GEMM_TRAFFIC
    assert len(t["source_sha256"]) in (0, 64)
    assert len(bench.K_SCORE_TC_TRAFFIC["source_sha256"]) in (0, 64)
    assert set(t["bytes_per_launch"]) == {f"{n}/{m}" for n in (128, 64)
                                          for m in ("bf16x2", "fp16x2", "bf16x2_real", "fp16x2_real")}
    # 6 H + 2.5 n log2 n + 4 S at 128 px, S = 1089: 0.628 Mflop
    assert abs(bench.flops_per_eval(128, 16) - 627716.0) < 1.0


def _run_reference(env_extra):
    import json
    import subprocess
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-images", "1", "--cpu-quats", "2"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    return [json.loads(l) for l in lines]


def test_reference_arm_line():
    """The oracle arm prints one line with the GPU arm's workload config and its own sample."""
    (line,) = _run_reference({"RANK": "0", "WORLD_SIZE": "1"})
    bench = _bench()
    import workloads
    cfg = workloads.get_config("throughput")
    wl = workloads.workload(cfg, n_img=0)
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["config"] == bench.workload_config(cfg, cfg.n_img, len(wl["quats"]) * len(wl["ctfs"]))
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert cb["sample"].startswith("1 images x 2 orientations")
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent():
    assert _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_cpu_fft_context_matches_oracle():
    """The context leg (the paper's FP32 Fourier variant on the host) computes the oracle's log P."""
    import numpy as np
    import oracle
    import workloads
    bench = _bench()
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=4)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:16]
    projs = oracle.projections(wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.npix, cfg.pixel_A)
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift, projs=projs)
    logp, seconds, threads = bench.run_cpu_fft_context(imgs, projs, cfg.max_shift, reps=2)
    assert seconds > 0 and threads >= 1
    np.testing.assert_allclose(logp, ref["logP"], rtol=0, atol=1e-4)
