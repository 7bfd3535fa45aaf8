"""bench.py on CPU: every name a function loads is bound somewhere (a
workload runner that reads another runner's variables fails only on the GPU
box otherwise), and the command lines the driver and DESIGN use parse."""
import ast
import builtins
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _unbound_names(src):
    tree = ast.parse(src)
    module = set()
    for n in tree.body:
        if isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            module.add(n.name)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            module.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, ast.Assign):
            module.update(t.id for t in n.targets if isinstance(t, ast.Name))
    bad = []
    for fn in (n for n in tree.body if isinstance(n, ast.FunctionDef)):
        bound = {a.arg for a in fn.args.args}
        for node in ast.walk(fn):
            if isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
                bound.add(node.id)
            elif isinstance(node, (ast.FunctionDef, ast.Lambda)):
                bound.update(a.arg for a in node.args.args)
                if isinstance(node, ast.FunctionDef):
                    bound.add(node.name)
            elif isinstance(node, (ast.Import, ast.ImportFrom)):
                bound.update((a.asname or a.name).split(".")[0] for a in node.names)
            elif isinstance(node, ast.ExceptHandler) and node.name:
                bound.add(node.name)
        for node in ast.walk(fn):
            if (isinstance(node, ast.Name) and isinstance(node.ctx, ast.Load) and node.id not in bound
                    and node.id not in module and not hasattr(builtins, node.id)):
                bad.append((fn.name, node.id, node.lineno))
    return bad


def test_bench_functions_load_only_bound_names():
    assert _unbound_names(open(os.path.join(ROOT, "bench.py")).read()) == []


@pytest.mark.parametrize("argv", [[], ["--impl", "reference"], ["--workload", "incore"], ["--workload", "gemm"],
                                  ["--workload", "batch"], ["--workload", "adjoint"], ["--workload", "jacobi3d"],
                                  ["--workload", "kmeans"], ["--tb", "10"], ["--rows", "131072", "--hbm-gib", "48"],
                                  ["--keep-stale", "--no-staged", "--user-kernel"]])
def test_bench_command_lines_parse(argv, monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    args = bench.parse()
    assert args.steps >= 1 and args.warmup >= 3
