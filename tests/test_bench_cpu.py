"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU and prints the JSON line the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


def test_reference_arm_under_torchrun_two_ranks():
    """Launched as the multi-GPU benchmark is (torchrun, two ranks; gloo on
    a machine without GPUs): rank 0 alone runs the oracle and prints one
    line with n_gpus = 2; the other rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_orbit_leg_bookkeeping_with_an_oracle_binding(monkeypatch):
    """The orbit leg's host logic (cases, shapes, rates, the hand-over of
    the first trajectory to the CPU comparison) on a stand-in binding whose
    srp_integrate runs the oracle's RK4 on trajectory 0: the comparison
    then reports a zero deviation for both force models."""
    import types

    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    from oracle import orbit as O
    monkeypatch.setattr(bench, "ORBIT_STEPS", 6)
    sizes = (19, 256, 256, 256, 256, 6)

    class MLP:
        def __init__(self, ctx, params=None, seed=0):
            n = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
            self.p = (np.random.default_rng(seed).normal(size=n) * 0.05).astype(np.float32)

        def params(self):
            return self.p.copy()

    def orbit_opts(**kw):
        o = types.SimpleNamespace(in_scale=np.ones(19), in_offset=np.zeros(19), out_mean=np.zeros(6),
                                  out_std=np.ones(6))
        o.__dict__.update(kw)
        return o

    def srp_integrate(ctx, o, z0, th, proxy=None, want_traj=False, dL_dzN=None):
        assert z0.shape[1] == 13 and th.shape == (z0.shape[0], o.n_theta)
        if o.model == 1:
            m = O.Model("cannonball", P=o.pressure, mass=o.mass, sun=o.sun)
        else:
            flat, off, layers = proxy.params(), 0, []
            for a, b in zip(sizes[:-1], sizes[1:]):
                layers.append((flat[off:off + a * b].reshape(b, a).astype(np.float64),
                               flat[off + a * b:off + a * b + b].astype(np.float64)))
                off += a * b + b
            m = O.Model("proxy", P=o.pressure, mass=o.mass, sun=o.sun, params=layers, scale=o.in_scale,
                        offset=o.in_offset, mean=o.out_mean, std=o.out_std)
        zN = np.zeros((z0.shape[0], 13))
        zN[0] = O.rk4(m, z0[0], th[0], o.dt, o.n_steps)
        return {"zN": zN}

    fake = types.SimpleNamespace(SRP_FM_CANNONBALL=1, SRP_FM_PROXY=2, MLP=MLP, orbit_opts=orbit_opts,
                                 srp_integrate=srp_integrate)
    summary, check = bench.orbit_leg(fake, None)
    assert summary["cannonball"]["trajectories"] == 1024 and summary["proxy"]["trajectories"] == 256
    assert all(summary[k]["rk4_steps_per_s"] > 0 for k in ("cannonball", "proxy"))
    res = bench.orbit_oracle(check)
    for k in ("cannonball", "proxy"):
        assert res[k]["end_position_rel_dev_vs_gpu"] == 0.0 and res[k]["rk4_steps_per_s"] > 0


def test_oracle_legs_beside_gradient_and_proxy():
    """The CPU legs that time the oracle beside the GPU gradient, proxy and
    256^2-ray tracer legs run on the host and report positive rates."""
    sys.path.insert(0, ROOT)
    import bench
    out = bench.oracle_extra_legs()
    assert out["grad"]["grad_evals_per_s"] > 0 and out["grad"]["cores"] >= 1
    assert out["surrogate"]["evals_per_s"] > 0
    assert out["tracer_evals_per_s_256sq_rays"]["value"] > 0


def test_gpu_arm_line_has_the_contract_keys():
    """The GPU arm's JSON line (built in run_ours, which needs a GPU to run)
    carries every key of the benchmark contract, checked on its source."""
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    fn = next(n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name == "run_ours")
    keys = set()
    for node in ast.walk(fn):
        if isinstance(node, ast.Assign) and any(isinstance(t, ast.Name) and t.id == "line" for t in node.targets) \
                and isinstance(node.value, ast.Dict):
            keys |= {k.value for k in node.value.keys if isinstance(k, ast.Constant)}
        if isinstance(node, ast.Subscript) and isinstance(node.value, ast.Name) and node.value.id == "line" \
                and isinstance(node.slice, ast.Constant):
            keys.add(node.slice.value)
    need = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "clocks", "cpu_baseline"}
    assert need <= keys, need - keys
