"""Shared helpers for the GPU parity tests (inputs from ``synth``, checks from ``tolerance``)."""

import numpy as np
import pytest
import torch

import synth

ALPHA, BETA = 1.5, 1.2


def dev():
    return torch.device("cuda:0")


def U(shape, tid, seed=0):
    return synth.uniform(shape, seed, tid, device=dev())


def I(shape, tid, seed=0, lo=-2, hi=2):
    return synth.integers(shape, seed, tid, lo=lo, hi=hi, device=dev())


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def kfmod():
    from paper_1305_1183_gb300 import kf
    kf.lib()
    return kf


@pytest.fixture(scope="session")
def built():
    from paper_1305_1183_gb300 import _build
    _build.build()
    return kfmod()
