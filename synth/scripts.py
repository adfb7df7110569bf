"""Seeded random scripts of elementary calls (workload generator, no arithmetic
of the method).

A script is a dict with "vars" (name -> ("v", n) | ("m", n, n) | ("s",)),
"inputs", "outputs" and "calls" [(op, [out], [ins], [scalars])] in the op
vocabulary of the library (AXPBY, SCAL, DOT, GEMV, GEMVT, GER).  Generation
rule: 6-10 calls drawn uniformly from AXPY (AXPBY with b = 1, in place),
SCAL (in place), DOT, GEMV, GEMVT and GER; each operand is an existing
variable of the right shape with probability 0.6, else a new input; GER
updates an existing matrix in place with probability 0.6, else writes a new
one; GEMV / GEMVT write a new vector with probability 0.6, else overwrite an
existing vector that is not their own input.  Scalars are uniform in [-1, 1)
(or drawn from {-1, 1, 2} for integer-exact scripts).
"""

from __future__ import annotations

import torch

from . import TID, _srl, bits

OPS = ["AXPY", "SCAL", "DOT", "GEMV", "GEMVT", "GER"]


class _Rng:
    def __init__(self, seed: int, stream: int):
        self.seed = seed
        self.stream = stream
        self.i = 0

    def u(self) -> float:
        b = bits(self.seed, TID["script"] * 1000 + self.stream, torch.tensor([self.i]))
        self.i += 1
        return float(_srl(b, 11)[0].item()) * 2.0 ** -53

    def choice(self, seq):
        return seq[min(int(self.u() * len(seq)), len(seq) - 1)]


def random_script(seed: int, index: int, n: int, ncalls: int | None = None, integer: bool = False) -> dict:
    rng = _Rng(seed, index)
    if ncalls is None:
        ncalls = 6 + min(int(rng.u() * 5), 4)
    vars_ = {"A0": ("m", n, n), "x0": ("v", n), "x1": ("v", n)}
    inputs = ["A0", "x0", "x1"]
    calls = []
    counter = {"v": 2, "m": 1, "s": 0}

    def new(kind):
        if kind == "v":
            name = f"x{counter['v']}"; vars_[name] = ("v", n)
        elif kind == "m":
            name = f"A{counter['m']}"; vars_[name] = ("m", n, n)
        else:
            name = f"d{counter['s']}"; vars_[name] = ("s",)
        counter[kind] += 1
        return name

    def pick(kind, exclude=()):
        pool = [k for k, v in vars_.items() if v[0] == kind and k not in exclude]
        if pool and rng.u() < 0.6:
            return rng.choice(sorted(pool))
        name = new(kind)
        inputs.append(name)
        return name

    def scalar():
        if integer:
            return float(rng.choice([-1.0, 1.0, 2.0]))
        return rng.u() * 2.0 - 1.0

    for _ in range(ncalls):
        op = rng.choice(OPS)
        if op == "AXPY":
            x = pick("v")
            y = pick("v", exclude=(x,))
            calls.append(("AXPBY", [y], [x, y], [scalar(), 1.0]))
        elif op == "SCAL":
            x = pick("v")
            calls.append(("SCAL", [x], [x], [scalar()]))
        elif op == "DOT":
            x = pick("v")
            y = pick("v")
            calls.append(("DOT", [new("s")], [x, y], []))
        elif op in ("GEMV", "GEMVT"):
            A = pick("m")
            x = pick("v")
            pool = [k for k, v in vars_.items() if v[0] == "v" and k != x]
            out = rng.choice(sorted(pool)) if (pool and rng.u() >= 0.6) else new("v")
            calls.append((op, [out], [A, x], [scalar(), 0.0]))
        else:  # GER
            A = pick("m")
            u = pick("v")
            v = pick("v")
            out = A if rng.u() < 0.6 else new("m")
            calls.append(("GER", [out], [A, u, v], [scalar()]))
    written = {c[1][0] for c in calls}
    outputs = sorted(written)
    return {"vars": vars_, "inputs": inputs, "outputs": outputs, "calls": calls, "n": n}
