"""Compile the CPU oracle (plain C) into oracle/_build/liboracle.so.

Test infrastructure: the shared library built here is loaded only by the tests, the
smoke check and the benchmark's CPU-baseline leg.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mpjsvd_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")          # binary64 working precision
OUT_EXT = os.path.join(OUT_DIR, "liboracle_ext.so")  # long double working precision


def _build_one(out, extra, force):
    hdr = os.path.join(HERE, "mpjsvd_oracle.h")
    if (not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC)
            and os.path.getmtime(out) >= os.path.getmtime(hdr)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    # -ffp-contract=off: no fused multiply-add contraction, so x86-64 and aarch64 round alike.
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"] + extra + \
        ["-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Build both oracle libraries if missing or stale; returns the binary64 one."""
    os.makedirs(OUT_DIR, exist_ok=True)
    _build_one(OUT_EXT, ["-DORC_LONG_DOUBLE"], force)
    return _build_one(OUT, [], force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
