"""Mutation check of the oracle's pins (test infrastructure, CPU only).

Plants one mistake at a time in a copy of oracle/ -- an arithmetic operator
swapped (+ -, * /, ** *), a unary minus dropped, a comparison loosened or
tightened (< <=, > >=), or a numeric constant changed (integers by one,
floats by 1%) -- and runs the oracle's CPU tests against each copy.  A
mistake that no test notices is printed as a survivor.  Survivors are either
equivalent (the changed code computes the same thing, e.g. a chunk size, a
boundary comparison met with probability zero, a slice past the end) or
below the statistical power of the sampler tests (1% constants); anything
else is a missing pin.

    python tests/oracle_mutation.py [oracle_file.py ...] [-j WORKERS]

Each worker holds its own copy of oracle/ and tests/ under
_build/oracle_mutation/ and links workloads/, the only other package the
oracle tests import.  Nothing here is imported by the tests or the library.
"""
import argparse
import ast
import copy
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "_build", "oracle_mutation")
TESTS = "tests/test_oracle_*.py tests/test_workloads.py"

SWAP = {ast.Add: ast.Sub, ast.Sub: ast.Add, ast.Mult: ast.Div, ast.Div: ast.Mult,
        ast.Pow: ast.Mult, ast.FloorDiv: ast.Mult}
CMP = {ast.Lt: ast.LtE, ast.LtE: ast.Lt, ast.Gt: ast.GtE, ast.GtE: ast.Gt}


def _sites(tree):
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.BinOp) and type(node.op) in SWAP:
            out.append(("binop", node))
        elif isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.USub):
            out.append(("neg", node))
        elif (isinstance(node, ast.Constant) and isinstance(node.value, (int, float))
              and not isinstance(node.value, bool)):
            out.append(("const", node))
        elif isinstance(node, ast.Compare) and len(node.ops) == 1 and type(node.ops[0]) in CMP:
            out.append(("cmp", node))
    return out


def _docstrings(tree):
    skip = set()
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.Module, ast.ClassDef)) and node.body:
            first = node.body[0]
            if isinstance(first, ast.Expr) and isinstance(first.value, ast.Constant):
                skip.add(id(first.value))
    return skip


def mutants(path):
    """(description, mutated source) for every mutation site of one file."""
    tree = ast.parse(open(path).read())
    skip = _docstrings(tree)
    base = _sites(tree)
    base_lines = ast.unparse(tree).splitlines()
    res = []
    for i, (kind, node) in enumerate(base):
        if id(node) in skip:
            continue
        t2 = copy.deepcopy(tree)
        n2 = _sites(t2)[i][1]
        if kind == "binop":
            n2.op = SWAP[type(n2.op)]()
            what = f"{type(node.op).__name__} -> {type(n2.op).__name__}"
        elif kind == "neg":
            n2.op = ast.UAdd()
            what = "unary minus dropped"
        elif kind == "cmp":
            n2.ops = [CMP[type(n2.ops[0])]()]
            what = f"{type(node.ops[0]).__name__} -> {type(n2.ops[0]).__name__}"
        else:
            v = node.value
            n2.value = v + 1 if isinstance(v, int) else (1e-3 if v == 0.0 else v * 1.01)
            what = f"constant {v!r} -> {n2.value!r}"
        try:
            text = ast.unparse(t2)
        except Exception:
            continue
        changed = [m for o, m in zip(base_lines, text.splitlines()) if o != m]
        res.append((f"line {node.lineno}: {what} | {changed[0].strip()[:100] if changed else ''}", text))
    return res


def _worker(k):
    d = os.path.join(WORK, f"w{k}")
    if os.path.isdir(d):
        shutil.rmtree(d)
    os.makedirs(d)
    os.symlink(os.path.join(ROOT, "workloads"), os.path.join(d, "workloads"))
    for name in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, name), os.path.join(d, name),
                        ignore=shutil.ignore_patterns("__pycache__"))
    return d


def _run(d, rel, text):
    target = os.path.join(d, "oracle", rel)
    original = open(os.path.join(ROOT, "oracle", rel)).read()
    open(target, "w").write(text)
    try:
        env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
        r = subprocess.run(f"timeout 300 python -m pytest {TESTS} -x -q -m 'not gpu' -p no:cacheprovider",
                           shell=True, cwd=d, capture_output=True, text=True, env=env)
        return r.returncode
    finally:
        open(target, "w").write(original)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("files", nargs="*")
    ap.add_argument("-j", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    a = ap.parse_args()
    files = a.files or sorted(f for f in os.listdir(os.path.join(ROOT, "oracle"))
                              if f.endswith(".py") and f != "__init__.py")
    jobs = [(f, desc, text) for f in files for desc, text in mutants(os.path.join(ROOT, "oracle", f))]
    print(f"{len(jobs)} mutants in {', '.join(files)}", flush=True)
    free = [_worker(k) for k in range(a.j)]
    # the unmutated copy must pass, or every mutant would count as caught
    base = files[0]
    if _run(free[0], base, open(os.path.join(ROOT, "oracle", base)).read()) != 0:
        raise SystemExit("the oracle tests fail on the unmutated copy")
    lock = threading.Lock()

    def task(job):
        with lock:
            d = free.pop()
        try:
            return job, _run(d, job[0], job[2])
        finally:
            with lock:
                free.append(d)

    survived = 0
    with ThreadPoolExecutor(a.j) as ex:
        for (f, desc, _), rc in ex.map(task, jobs):
            if rc == 0:
                survived += 1
                print(f"survived  {f} {desc}", flush=True)
    print(f"{survived} of {len(jobs)} mutants survived")


if __name__ == "__main__":
    main()
