"""Sequential FP64 interpreter for scripts of elementary calls (test infrastructure only).

The paper's script (Section 3.4, Listing 1) declares typed variables, marks
inputs, calls elementary functions in order and returns outputs; the calls'
order and data dependencies define the result (Section 3.1).  This module
evaluates such a script call by call in float64, with the elementaries of
``kf_oracle.c``; fusion must not change its result.

A script is a list of calls ``(op, outs, ins, scalars)`` over named variables.
Op semantics (BLAS conventions):

  AXPBY  out = a*x + b*y                 ins (x, y)      scalars (a, b)
  SCAL   out = a*x                       ins (x,)        scalars (a,)
  DOT    out = x . y   (a scalar)        ins (x, y)
  VADD   out = w + y + z                 ins (w, y, z)
  GEMV   out = a*A x + b*y0              ins (A, x[, y0]) scalars (a, b)
  GEMVT  out = a*A^T y + b*x0            ins (A, y[, x0]) scalars (a, b)
  GER    out = A + a*u v^T               ins (A, u, v)   scalars (a,)
  MADD   out = A + B                     ins (A, B)
"""

from __future__ import annotations

import numpy as np

from . import axpby, dot, gemv, gemvt, ger, madd, vadd3


def run(calls, env: dict) -> dict:
    """Evaluate ``calls`` on a copy of ``env`` (name -> array or float).
    Returns the final environment, all values in float64."""
    E = {k: (np.asarray(v, dtype=np.float64).copy() if not np.isscalar(v) else float(v))
         for k, v in env.items()}
    for op, outs, ins, sc in calls:
        sc = list(sc) + [0.0] * (2 - len(sc))
        a, b = float(sc[0]), float(sc[1])
        X = [E[i] for i in ins]
        if op == "AXPBY":
            r = axpby(a, X[0], b, X[1])
        elif op == "SCAL":
            r = axpby(a, X[0], 0.0, X[0])
        elif op == "DOT":
            r = dot(X[0], X[1])
        elif op == "VADD":
            r = vadd3(X[0], X[1], X[2])
        elif op == "GEMV":
            r = gemv(X[0], X[1], a, b, X[2] if len(X) > 2 else None)
        elif op == "GEMVT":
            r = gemvt(X[0], X[1], a, b, X[2] if len(X) > 2 else None)
        elif op == "GER":
            r = ger(X[0], X[1], X[2], a)
        elif op == "MADD":
            r = madd(X[0], X[1])
        else:
            raise ValueError(f"unknown op {op}")
        E[outs[0]] = r
    return E
