"""Compiles the C part of the oracle (``direct.c``) into ``oracle/_direct.so``.

Test infrastructure only.  Called by ``__graft_entry__.build()`` and lazily by
``oracle.direct.direct_sum_c``.
"""
from __future__ import annotations

import os
import subprocess


def build() -> str:
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "direct.c")
    out = os.path.join(here, "_direct.so")
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared",
                           "-fPIC", src, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out
