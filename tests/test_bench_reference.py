"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on
CPU and prints one JSON line with the fields the contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_ball_oracle_leg_bounds_points_of_the_ball():
    """The CPU leg of the bench's l2-ball config states the workload on the
    oracle side (interval bounds over the ball, its own masks) and bounds a
    sample of it: every bound is below the network at points of the ball
    (weak duality; the leg's subdomains are splits of the same ball)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import l2
    wl = dict(bench.make_workload("base", 0, B=4, T=5), ball_eps=0.1)
    on, lbk, ubk, masks = bench.oracle_problem(wl)
    assert lbk.shape == (1, 3172) and masks.shape == (4, 3172)
    out = bench.oracle_run(on, wl, lbk, ubk, masks[:2])
    c = bench.ball_centre(wl)[0].astype(np.float64)
    vals = on.evaluate(l2.ball_points(c, 0.1, 64, seed=2))
    assert np.all(np.isfinite(out)) and np.all(out[:, None] <= vals[None, :] + 1e-9)
