"""Static checks of the GPU test modules, which a machine without a GPU skips
at import: every name a parametrize decorator lists is an argument of the
test it decorates, and every module compiles."""
import ast
import glob
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(HERE, "test_gpu_*.py")))
                         + [os.path.join(HERE, "test_zz_no_alloc.py")])
def test_gpu_module_parametrize_matches_signatures(path):
    tree = ast.parse(open(path).read(), filename=path)
    compile(tree, path, "exec")
    for node in tree.body:
        if not isinstance(node, ast.FunctionDef):
            continue
        args = {a.arg for a in node.args.args}
        for d in node.decorator_list:
            if isinstance(d, ast.Call) and getattr(d.func, "attr", "") == "parametrize":
                names = [n.strip() for n in d.args[0].value.split(",")]
                assert set(names) <= args, (node.name, names)
