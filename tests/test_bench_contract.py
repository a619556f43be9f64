"""The benchmark's output contract, checked on the source (no GPU): the JSON line of each arm carries
every key its consumers read, and the timed region's rate comes from the slowest rank."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MAIN_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline"}
ROOFLINE_KEYS = {"bound", "achieved", "peak", "unit", "frac", "traffic"}
E2E_KEYS = {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
CPU_KEYS = {"value", "unit", "cores", "kind", "sample"}


def _dict_assigned(fn, name):
    for node in ast.walk(fn):
        if isinstance(node, ast.Assign) and any(isinstance(t, ast.Name) and t.id == name for t in node.targets):
            if isinstance(node.value, ast.Dict):
                return node.value
    raise AssertionError(f"no dict literal assigned to {name!r} in {fn.name}")


def _keys(d):
    return {k.value for k in d.keys if isinstance(k, ast.Constant)}


def _sub(d, key):
    for k, v in zip(d.keys, d.values):
        if isinstance(k, ast.Constant) and k.value == key:
            return v
    raise AssertionError(key)


def _functions():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    return {n.name: n for n in tree.body if isinstance(n, ast.FunctionDef)}


def _returned_dict(fn):
    for node in ast.walk(fn):
        if isinstance(node, ast.Return) and isinstance(node.value, ast.Dict):
            return node.value
    raise AssertionError(f"{fn.name} returns no dict literal")


def _config_call(line):
    c = _sub(line, "config")
    assert isinstance(c, ast.Call) and isinstance(c.func, ast.Name), "config comes from one helper"
    return c


def test_main_line_keys():
    fns = _functions()
    line = _dict_assigned(fns["main"], "line")
    assert MAIN_KEYS <= _keys(line)
    assert E2E_KEYS <= _keys(_sub(line, "e2e"))
    assert CPU_KEYS <= _keys(_dict_assigned(fns["main"], "cpu"))
    # the roofline object is built by update_roofline (the headline's dominant kernel), or by oz_roofline (A G)
    assert ROOFLINE_KEYS <= _keys(_returned_dict(fns["update_roofline"]))
    assert ROOFLINE_KEYS <= _keys(_returned_dict(fns["oz_roofline"]))
    assert ROOFLINE_KEYS <= _keys(_returned_dict(fns["fp64_roofline"]))
    assert "workload" in _keys(_returned_dict(fns["workload_config"]))


def test_reference_line_keys():
    fns = _functions()
    line = _dict_assigned(fns["run_reference"], "line")
    assert (MAIN_KEYS - {"roofline", "gpu_launches", "clocks"}) | {"impl"} <= _keys(line)
    assert CPU_KEYS <= _keys(_sub(line, "cpu_baseline"))
    assert E2E_KEYS <= _keys(_sub(line, "e2e"))


def test_both_arms_name_the_same_workload():
    """Identical config dicts: both arms build theirs with the same helper and the same arguments."""
    fns = _functions()
    main_cfg = _config_call(_dict_assigned(fns["main"], "line"))
    ref_cfg = _config_call(_dict_assigned(fns["run_reference"], "line"))
    assert main_cfg.func.id == ref_cfg.func.id == "workload_config"
    assert [ast.unparse(a) for a in main_cfg.args] == [ast.unparse(a) for a in ref_cfg.args]


def test_rates_use_the_slowest_rank():
    src = ast.unparse(_functions()["main"])  # literals are normalised: 1e3 reads back as 1000.0
    assert "ms_max = ranks.max_over_ranks(ms, world, 'cuda')" in src
    assert "value = ranks.whole_job_rate(args.steps, world, ms_max / 1000.0)" in src
    assert "ranks.whole_job_rate(args.steps, world, ranks.max_over_ranks(e2e_s, world, 'cuda'))" in src
