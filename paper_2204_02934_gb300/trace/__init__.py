"""GPU activity traces for measurement: the kernels, memsets and copies a
stretch of host code runs on the device, each with its device start and end
time, and the idle gaps between them.

Records come from CUPTI's activity API through a small C++ shim
(`cupti_trace.cpp`), built on first use into `libmis2_trace.so` with g++
against the CUDA toolkit's CUPTI.  Measurement only: the library's compute
path never loads it.

    from paper_2204_02934_gb300 import trace
    with trace.GpuTrace() as t:
        ...                          # device work
    print(trace.summary(t.records))
"""
from __future__ import annotations

import ctypes
import glob
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cupti_trace.cpp")
LIB = os.path.join(HERE, "libmis2_trace.so")


def _cuda_home() -> str:
    return os.environ.get("CUDA_HOME") or "/usr/local/cuda"


def _cupti_dir() -> str:
    home = _cuda_home()
    for pat in ("targets/*/lib/libcupti.so", "extras/CUPTI/lib64/libcupti.so", "lib64/libcupti.so"):
        hits = sorted(glob.glob(os.path.join(home, pat)))
        if hits:
            return os.path.dirname(hits[0])
    raise RuntimeError(f"CUPTI not found under {home}")


def build(force: bool = False) -> str:
    """Compile the shim (if missing or older than its source); returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    libdir = _cupti_dir()
    tmp = LIB + ".tmp"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", os.path.join(_cuda_home(), "include"), SRC,
                    "-o", tmp, "-L", libdir, "-lcupti", "-Wl,-rpath," + libdir], check=True)
    os.replace(tmp, LIB)
    return LIB


def parse(path: str) -> list[dict]:
    """Records of a trace file, in order of device start time."""
    out = []
    for line in open(path):
        kind, start, end, stream, name = line.rstrip("\n").split(" ", 4)
        out.append({"kind": {"K": "kernel", "S": "memset", "C": "memcpy"}[kind], "start_ns": int(start),
                    "end_ns": int(end), "stream": int(stream), "name": name})
    out.sort(key=lambda r: r["start_ns"])
    return out


class GpuTrace:
    """Context manager recording the device activity of its body (the device
    is synchronised on entry and exit); `records` holds it afterwards."""

    def __init__(self):
        self.records: list[dict] = []

    def __enter__(self):
        import torch

        torch.cuda.synchronize()
        self._lib = ctypes.CDLL(build())
        fd, self._path = tempfile.mkstemp(suffix=".trace")
        os.close(fd)
        rc = self._lib.mis2_trace_start(self._path.encode())
        if rc != 0:
            raise RuntimeError(f"mis2_trace_start failed ({rc})")
        return self

    def __exit__(self, *exc):
        import torch

        torch.cuda.synchronize()
        self._lib.mis2_trace_stop()
        self.records = parse(self._path)
        os.unlink(self._path)
        return False


def short_name(name: str) -> str:
    """A readable kernel name: the identifier inside a mangled mis2:: name."""
    if name.startswith("_ZN4mis2"):
        rest = name[len("_ZN4mis2"):]
        digits = ""
        while rest and rest[0].isdigit():
            digits += rest[0]
            rest = rest[1:]
        if digits:
            return rest[:int(digits)]
    return name.split("(")[0][:48]


def summary(records: list[dict]) -> dict:
    """Span from the first start to the last end, time covered by at least
    one operation, idle time in between, and per operation name its count and
    summed duration (operations launched with programmatic dependent launch
    overlap their predecessor, so durations can add up to more than the
    covered time)."""
    if not records:
        return {"ops": 0}
    t0 = records[0]["start_ns"]
    covered, cur_s, cur_e = 0, records[0]["start_ns"], records[0]["end_ns"]
    for r in records[1:]:
        if r["start_ns"] > cur_e:
            covered += cur_e - cur_s
            cur_s, cur_e = r["start_ns"], r["end_ns"]
        else:
            cur_e = max(cur_e, r["end_ns"])
    covered += cur_e - cur_s
    span = max(r["end_ns"] for r in records) - t0
    per = {}
    for r in records:
        k = short_name(r["name"]) if r["kind"] == "kernel" else r["name"].split("_")[0]
        c = per.setdefault(k, [0, 0])
        c[0] += 1
        c[1] += r["end_ns"] - r["start_ns"]
    return {"ops": len(records), "kernels": sum(r["kind"] == "kernel" for r in records),
            "span_us": span / 1e3, "covered_us": covered / 1e3, "idle_us": (span - covered) / 1e3,
            "per_name": {k: {"count": v[0], "us": round(v[1] / 1e3, 1)} for k, v in
                         sorted(per.items(), key=lambda kv: -kv[1][1])}}
