"""bench.py's short batched and served runs reported under 'forms' in the default line:
the sub-runs get their own workload, step counts and no oracle baseline, the caller's
arguments are left as they were, and a failing sub-run is reported in place of its numbers
instead of stopping the headline line (CPU: the two runs are replaced by stand-ins)."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_forms_use_their_own_settings_and_isolate_failures(monkeypatch):
    import bench

    seen = []

    def batch(a, emit=True):
        seen.append(("batched", a.workload, a.steps, a.warmup, a.skip_cpu, a.tune, emit))
        return {"metric": bench.BATCH_METRIC, "value": 10.0, "unit": "graphs/s",
                "ms_per_step": 5.0, "steps": a.steps, "warmup": a.warmup,
                "config": {"workload": a.workload}, "roofline": {"frac": 0.25},
                "clocks": {"sm_mhz": 2070.0}, "unlisted": 1}

    def serve(a, emit=True):
        seen.append(("served", a.workload, a.steps, a.warmup, a.skip_cpu, a.tune, emit))
        raise RuntimeError("no device")

    monkeypatch.setattr(bench, "run_batch", batch)
    monkeypatch.setattr(bench, "run_serve", serve)
    args = argparse.Namespace(workload="lfr26", steps=10, warmup=5, tune=True, skip_cpu=False,
                              mode="mg", k=8, no_forms=False)
    out = bench.measure_forms(args)
    assert seen == [("batched", "sbm256", 3, 3, True, False, False),
                    ("served", "serve", 1, 3, True, False, False)]
    assert (args.workload, args.steps, args.warmup, args.tune, args.skip_cpu) == \
        ("lfr26", 10, 5, True, False)
    b = out["batched"]
    assert b["value"] == 10.0 and b["roofline_frac"] == 0.25 and "unlisted" not in b
    assert b["config"] == {"workload": "sbm256"}
    assert out["served"]["error"] == "RuntimeError: no device"
    assert set(out) == {"batched", "served"}
