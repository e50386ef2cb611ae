"""Checkpoint and resume of a run: the nodal state (u, v), the time, the step
count and the problem description, in one .npz file.

The library keeps no state across gdg_step calls that the result depends on
(each call starts from the nodal state it is given, and every kernel is
deterministic), so a run resumed from a checkpoint in a new context -- or a
new process -- continues exactly as the original run would have.
"""
import json

import numpy as np

from . import gdg

_ARRAYS = ("x_nodes", "y_nodes", "c2_nodes")


def save(path, u, v, t, step, problem):
    """Write u, v (device tensors or arrays), t, step and the keyword
    arguments of gdg.make_problem (`problem`, a dict) to `path`."""
    arrays = {k: np.ascontiguousarray(problem[k], dtype=np.float64) for k in _ARRAYS if problem.get(k) is not None}
    scalars = {k: (list(v_) if isinstance(v_, tuple) else v_) for k, v_ in problem.items() if k not in _ARRAYS}
    as_np = lambda a: a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    np.savez(path, u=as_np(u), v=as_np(v), t=np.float64(t), step=np.int64(step),
             problem=np.array(json.dumps(scalars)), **{"arr_" + k: a for k, a in arrays.items()})


def load(path):
    """(u, v, t, step, problem) with u, v as float64 numpy arrays and
    `problem` the keyword arguments for gdg.make_problem."""
    with np.load(path) as f:
        problem = json.loads(str(f["problem"]))
        for k in _ARRAYS:
            if "arr_" + k in f:
                problem[k] = f["arr_" + k].copy()
        for k in ("n", "lo", "hi", "bc"):
            if k in problem and isinstance(problem[k], list):
                problem[k] = tuple(problem[k])
        return f["u"].copy(), f["v"].copy(), float(f["t"]), int(f["step"]), problem


def make_problem(problem):
    """gdg.make_problem from a checkpoint's problem description."""
    return gdg.make_problem(**problem)
