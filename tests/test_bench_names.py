"""Static check (no GPU) of the benchmark and entry-point scripts: every name a
function reads or deletes is bound somewhere it can see (its own scope, an
enclosing function, the module, or the builtins). A stale name in a code path
that only the full GPU run reaches (for instance a `del` of a variable that a
refactor removed) otherwise surfaces only after every measurement has run."""

import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ["bench.py", "__graft_entry__.py", os.path.join("paper_1707_09177_gb300", "__init__.py"),
         os.path.join("paper_1707_09177_gb300", "build.py")]


def _bound_in(node):
    """Names bound directly in the scope of `node` (not in nested functions)."""
    names = set()
    if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
        a = node.args
        for arg in a.posonlyargs + a.args + a.kwonlyargs:
            names.add(arg.arg)
        if a.vararg:
            names.add(a.vararg.arg)
        if a.kwarg:
            names.add(a.kwarg.arg)
    body = node.body if isinstance(node.body, list) else [node.body]
    stack = list(body)
    while stack:
        n = stack.pop()
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(n.name)
            stack.extend(n.decorator_list)
            continue
        if isinstance(n, ast.Lambda):
            continue
        if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store):
            names.add(n.id)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            for al in n.names:
                names.add((al.asname or al.name).split(".")[0])
        elif isinstance(n, ast.ExceptHandler) and n.name:
            names.add(n.name)
        elif isinstance(n, (ast.Global, ast.Nonlocal)):
            names.update(n.names)
        elif isinstance(n, ast.NamedExpr):
            names.add(n.target.id)
        stack.extend(ast.iter_child_nodes(n))
    return names


def _used_in(node):
    """(name, line, how) for every Name read or deleted directly in the scope of
    `node`, and the nested function scopes found there."""
    used, nested = [], []
    body = node.body if isinstance(node.body, list) else [node.body]
    stack = list(body)
    while stack:
        n = stack.pop()
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
            nested.append(n)
            if not isinstance(n, ast.Lambda):
                stack.extend(n.decorator_list)
            stack.extend(n.args.defaults + [d for d in n.args.kw_defaults if d is not None])
            continue
        if isinstance(n, ast.ClassDef):
            nested.append(n)
            continue
        if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Load, ast.Del)):
            used.append((n.id, n.lineno, "deleted" if isinstance(n.ctx, ast.Del) else "read"))
        stack.extend(ast.iter_child_nodes(n))
    return used, nested


def unbound_names(source):
    tree = ast.parse(source)
    module_names = _bound_in(tree) | set(dir(builtins)) | {"__file__", "__name__", "__doc__"}
    problems = []

    def visit(scope, visible):
        mine = _bound_in(scope) if not isinstance(scope, ast.ClassDef) else set()
        seen = visible | mine
        used, nested = _used_in(scope)
        for name, line, how in used:
            if name not in seen:
                problems.append("%s but never bound: %s (line %d)" % (how, name, line))
        for n in nested:
            visit(n, seen)

    _, top = _used_in(tree)
    for n in top:
        visit(n, module_names)
    return problems


@pytest.mark.parametrize("rel", FILES)
def test_every_name_is_bound(rel):
    with open(os.path.join(ROOT, rel)) as f:
        src = f.read()
    assert unbound_names(src) == []


def test_the_check_finds_a_stale_delete():
    src = ("def main():\n    out = 1\n    host_out = 2\n    del out, dev_in, host_out\n")
    assert unbound_names(src) == ["deleted but never bound: dev_in (line 4)"]


def test_the_check_accepts_closures_and_comprehensions():
    src = ("import os\nX = 1\n\ndef f(a, *b, c=2, **d):\n    y = [i for i in b]\n"
           "    def g():\n        return a + X + len(y) + os.sep.count('/')\n    return g\n")
    assert unbound_names(src) == []
