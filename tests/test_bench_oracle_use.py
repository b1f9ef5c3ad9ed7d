"""The benchmark may run the oracle in two places only: its reference arm and the
CPU-baseline leg of the GPU arm (the block under `not args.no_cpu_baseline`).
Every other leg measures the product alone; GPU-oracle equality is the parity
tests' job."""

import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _parents(tree):
    par = {}
    for node in ast.walk(tree):
        for child in ast.iter_child_nodes(node):
            par[child] = node
    return par


def test_oracle_only_in_reference_arm_and_cpu_baseline():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    par = _parents(tree)
    uses = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
            uses.append(node)
        if isinstance(node, ast.ImportFrom) and node.module and node.module.split(".")[0] == "oracle":
            uses.append(node)
    assert uses
    for node in uses:
        chain, p = [], par.get(node)
        while p is not None:
            chain.append(p)
            p = par.get(p)
        funcs = [p.name for p in chain if isinstance(p, ast.FunctionDef)]
        assert funcs, f"module-level oracle import at line {node.lineno}"
        if funcs[0] in ("reference_arm", "_oracle_worker"):
            continue
        assert funcs[0] == "gpu_arm", f"oracle imported in {funcs[0]} (line {node.lineno})"
        guards = [ast.unparse(p.test) for p in chain if isinstance(p, ast.If)]
        assert any("no_cpu_baseline" in g for g in guards), f"oracle outside the CPU-baseline leg (line {node.lineno})"
    # the all-cores baseline runs the oracle in spawned workers (a module-level function,
    # so that it can be pickled): it is reached only from the CPU-baseline leg
    calls = {"_oracle_worker": [], "cpu_all_cores": []}
    for node in ast.walk(tree):
        if isinstance(node, ast.Name) and node.id in calls and not isinstance(par.get(node), ast.FunctionDef):
            calls[node.id].append(node)
    for node in calls["_oracle_worker"]:
        chain, p = [], par.get(node)
        while p is not None:
            chain.append(p)
            p = par.get(p)
        funcs = [p.name for p in chain if isinstance(p, ast.FunctionDef)]
        assert funcs and funcs[0] == "cpu_all_cores", f"oracle worker used in {funcs} (line {node.lineno})"
    assert calls["cpu_all_cores"]
    for node in calls["cpu_all_cores"]:
        chain, p = [], par.get(node)
        while p is not None:
            chain.append(p)
            p = par.get(p)
        funcs = [p.name for p in chain if isinstance(p, ast.FunctionDef)]
        guards = [ast.unparse(p.test) for p in chain if isinstance(p, ast.If)]
        assert funcs and funcs[0] == "gpu_arm" and any("no_cpu_baseline" in g for g in guards), \
            f"all-cores oracle baseline outside the CPU-baseline leg (line {node.lineno})"


def test_product_package_never_imports_the_oracle():
    """Nothing in the package (binding, trainer, build) imports, loads or links the
    oracle: the product path is the CUDA library or an error."""
    pkg = os.path.join(ROOT, "paper_2010_14333_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if not fn.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                continue
            path = os.path.join(dirpath, fn)
            src = open(path, errors="replace").read()
            if fn.endswith(".py"):
                for node in ast.walk(ast.parse(src)):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert not (node.module or "").startswith("oracle"), path
            assert "rx_oracle" not in src and "liborx" not in src, path


def test_reference_arm_prints_its_line():
    """The reference arm (the FP64 oracle on the host cores) runs one step of the
    workload's buffers and prints one JSON line with the fields the launch contract
    asks of it: impl, the GPU arm's metric and unit, its own cpu_baseline and a zero-copy
    e2e block whose value is the line's."""
    import json
    import subprocess
    import sys

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GSa/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GSa/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert 0 < d["ber"] < 0.02


def test_reference_arm_under_two_ranks():
    """Launched as the multi-GPU bench is (torch.distributed.run, two ranks), the
    reference arm runs on rank 0 alone: one line, every rank exits 0."""
    import json
    import socket
    import subprocess
    import sys

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
