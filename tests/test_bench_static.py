"""bench.py's GPU-only code paths cannot run here; this checks statically that every name a
function reads is bound somewhere (a parameter, an assignment, an import, a module-level
definition or a builtin), so a stale variable fails without a GPU instead of when the path runs."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _walk_scope(node):
    """The nodes of one scope: nested function bodies are not entered (their names are)."""
    todo = list(ast.iter_child_nodes(node))
    while todo:
        n = todo.pop()
        yield n
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
            todo.extend(n.args.defaults + n.args.kw_defaults if isinstance(n, ast.Lambda) else n.decorator_list)
            continue
        todo.extend(ast.iter_child_nodes(n))


def _bound_names(node, walk=ast.walk):
    names = set()
    for n in walk(node):
        if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            names.add(n.id)
        elif isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(n.name)
        elif isinstance(n, ast.arg):
            names.add(n.arg)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            for a in n.names:
                names.add((a.asname or a.name).split(".")[0])
        elif isinstance(n, ast.ExceptHandler) and n.name:
            names.add(n.name)
        elif isinstance(n, (ast.Global, ast.Nonlocal)):
            names.update(n.names)
    return names


def _check_scope(fn, enclosing, missing):
    """Names read in function `fn` (not in its nested functions) must be bound in fn or in an
    enclosing scope; nested functions are checked with fn's names added."""
    known = enclosing | _bound_names(fn, _walk_scope)
    for n in _walk_scope(fn):
        if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load) and n.id not in known:
            missing.append(f"{fn.name}:{n.lineno}:{n.id}")
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef)):
            _check_scope(n, known, missing)


def test_bench_has_no_unbound_names():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    module_names = _bound_names(tree, _walk_scope) | set(dir(builtins)) | {"__file__", "__name__"}
    missing = []
    for fn in _walk_scope(tree):
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            _check_scope(fn, module_names, missing)
    assert not missing, missing
