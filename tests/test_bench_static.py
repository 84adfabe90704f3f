"""bench.py on the CPU: every name a function reads is bound in that
function, at module level or as a builtin (the GPU legs cannot run here,
so a stale name in one of them would otherwise surface only on a GPU), and
the argument parser accepts the documented flags."""
import ast
import builtins
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _module_names(tree):
    names = set()
    for n in tree.body:
        if isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            names.add(n.name)
        elif isinstance(n, ast.Assign):
            names |= {t.id for t in n.targets if isinstance(t, ast.Name)}
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            names |= {(a.asname or a.name).split(".")[0] for a in n.names}
    return names


def _bound_in(fn):
    bound = {a.arg for a in fn.args.args + fn.args.kwonlyargs}
    for node in ast.walk(fn):
        if isinstance(node, ast.Name) and isinstance(node.ctx, ast.Store):
            bound.add(node.id)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            bound |= {(a.asname or a.name).split(".")[0] for a in node.names}
        elif isinstance(node, (ast.FunctionDef, ast.Lambda)):
            if isinstance(node, ast.FunctionDef):
                bound.add(node.name)
            bound |= {a.arg for a in node.args.args}
        elif isinstance(node, ast.ExceptHandler) and node.name:
            bound.add(node.name)
    return bound


def test_bench_functions_read_only_bound_names():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    module = _module_names(tree)
    problems = {}
    for fn in (n for n in tree.body if isinstance(n, ast.FunctionDef)):
        used = {n.id for n in ast.walk(fn) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
        missing = sorted(u for u in used - _bound_in(fn) - module if not hasattr(builtins, u))
        if missing:
            problems[fn.name] = missing
    assert not problems, problems


def test_bench_help_lists_the_flags():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--k1", "--no-graph", "--no-tune",
                 "--e2e-steps", "--precision"):
        assert flag in out.stdout, flag
