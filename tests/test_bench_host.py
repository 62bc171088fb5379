"""bench.py on the host (no GPU): every global name its functions use is defined, the recorded
traffic tables are well formed, and the algorithmic work per evaluation is what DESIGN states."""
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


def test_traffic_tables_and_work_per_eval():
    bench = _bench()
    assert len(bench.K_SCORE_TRAFFIC["source_sha256"]) == 64 and bench.K_SCORE_TRAFFIC["bytes_per_pair"] > 0
    t = bench.K_SCORE_GEMM_TRAFFIC
    assert len(t["source_sha256"]) == 64
    assert set(t["bytes_per_launch"]) == {f"{n}/{m}" for n in (128, 64)
                                          for m in ("bf16x2", "fp16x2", "bf16x2_real", "fp16x2_real")}
    # 6 H + 2.5 n log2 n + 4 S at 128 px, S = 1089: 0.628 Mflop
    assert abs(bench.flops_per_eval(128, 16) - 627716.0) < 1.0
