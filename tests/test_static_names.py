"""Static checks on the CPU of code whose GPU paths cannot run here
(bench.py, the entry points, the package's Python modules): every name a
function reads is bound in that function, at module level or as a builtin
-- a stale name in a GPU leg would otherwise surface only on a GPU -- and
bench.py's argument parser accepts the documented flags."""
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
        elif isinstance(n, (ast.Assign, ast.AnnAssign)):
            targets = n.targets if isinstance(n, ast.Assign) else [n.target]
            for t in targets:
                names |= {e.id for e in ast.walk(t) if isinstance(e, ast.Name)}
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            names |= {(a.asname or a.name).split(".")[0] for a in n.names}
    return names


def _bound_in(fn):
    bound = {a.arg for a in fn.args.args + fn.args.kwonlyargs + fn.args.posonlyargs}
    bound |= {a.arg for a in (fn.args.vararg, fn.args.kwarg) if a is not None}
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


def _functions(tree):
    for n in tree.body:
        if isinstance(n, ast.FunctionDef):
            yield n.name, n
        elif isinstance(n, ast.ClassDef):
            for m in n.body:
                if isinstance(m, ast.FunctionDef):
                    yield f"{n.name}.{m.name}", m


# the scripts and the package modules whose GPU paths cannot run here
FILES = ["bench.py", "__graft_entry__.py"] + [
    os.path.join("paper_2601_11626_gb300", f)
    for f in ("csvd.py", "sharded.py", "tune.py", "paper_shapes.py", "diagnostics.py", "synth.py")]


def test_functions_read_only_bound_names():
    problems = {}
    for f in FILES:
        tree = ast.parse(open(os.path.join(ROOT, f)).read())
        module = _module_names(tree)
        for name, fn in _functions(tree):
            used = {n.id for n in ast.walk(fn)
                    if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
            missing = sorted(u for u in used - _bound_in(fn) - module if not hasattr(builtins, u))
            if missing:
                problems[f"{f}:{name}"] = missing
    assert not problems, problems


def test_bench_help_lists_the_flags():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--k1", "--no-graph", "--no-tune",
                 "--e2e-steps", "--precision"):
        assert flag in out.stdout, flag
