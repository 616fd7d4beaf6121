"""Compile a mechanism into a loadable artefact (cubin + metadata).

    build_mechanism(mech_dict) -> artefact directory

The directory holds ``mech.cu`` (the translation unit: device math, the
generated body, the kernel templates), ``mech.cubin`` (sm_103a), ``meta.txt``
(read by the C runtime) and ``meta.json`` (op counts, registers, spills).
Artefacts are cached by a digest of the mechanism, the compile options and
the hand-written templates.
"""
from __future__ import annotations

import hashlib
import json
import os
import re
import shutil
import subprocess
import time

from . import emit, mech as qmech, model as qmodel

PKG = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(PKG, "csrc")
REPO = os.path.dirname(PKG)
DEFAULT_ROOT = os.path.join(REPO, "build", "mech")
NVCC = os.environ.get("QSS_NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
TEMPLATES = ["qss_device.cuh", "qss_exp_table.inc", "qss_kernels.cuh", "qss_newton.cuh"]
COMPILER_VERSION = "1"


def _template_digest():
    h = hashlib.sha256(COMPILER_VERSION.encode())
    for t in TEMPLATES:
        p = os.path.join(CSRC, t)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    for f in ("emit.py", "model.py", "expr.py", "mech.py", "graph.py"):
        h.update(open(os.path.join(os.path.dirname(__file__), f), "rb").read())
    return h.hexdigest()[:12]


def artefact_key(mech: dict, block: int = 128, defines=()) -> str:
    h = hashlib.sha256(json.dumps(mech, sort_keys=True).encode())
    h.update(f"{block}|{sorted(defines)}|{_template_digest()}".encode())
    return h.hexdigest()[:20]


def build_mechanism(mech: dict, root: str = DEFAULT_ROOT, block: int = 128, defines=(),
                    force: bool = False, verbose: bool = False) -> str:
    key = artefact_key(mech, block, defines)
    out = os.path.join(root, f"{mech.get('name', 'mech')}_{key}")
    if not force and os.path.exists(os.path.join(out, "mech.cubin")) and \
            os.path.exists(os.path.join(out, "meta.txt")):
        return out
    t0 = time.time()
    ir = qmech.parse(mech)
    model = qmodel.build_model(ir)
    src, meta = emit.emit_mechanism_source(model)
    tmp = out + ".tmp%d" % os.getpid()
    os.makedirs(tmp, exist_ok=True)
    with open(os.path.join(tmp, "mech_body.inc"), "w") as f:
        f.write(src)
    tu = ['#include "qss_device.cuh"', '#include "mech_body.inc"', '#include "qss_kernels.cuh"']
    if os.path.exists(os.path.join(CSRC, "qss_newton.cuh")):
        tu.append('#include "qss_newton.cuh"')
    with open(os.path.join(tmp, "mech.cu"), "w") as f:
        f.write("\n".join(tu) + "\n")
    t1 = time.time()
    cmd = [NVCC, "-cubin", *ARCH, "-O3", "-lineinfo", "-Xptxas", "-v", f"-DQSS_BLOCK={block}",
           *[f"-D{d}" for d in defines], "-I", CSRC, "-I", tmp, "-o", os.path.join(tmp, "mech.cubin"),
           os.path.join(tmp, "mech.cu")]
    p = subprocess.run(cmd, capture_output=True, text=True)
    log = p.stdout + p.stderr
    with open(os.path.join(tmp, "build.log"), "w") as f:
        f.write(" ".join(cmd) + "\n" + log)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {mech.get('name')}:\n{log[-4000:]}")
    meta["kernels"] = _parse_ptxas(log)
    meta["block"] = block
    meta["defines"] = list(defines)
    meta["codegen_s"] = round(t1 - t0, 3)
    meta["nvcc_s"] = round(time.time() - t1, 3)
    meta["artefact_key"] = key
    with open(os.path.join(tmp, "meta.json"), "w") as f:
        json.dump(meta, f, indent=1)
    with open(os.path.join(tmp, "meta.txt"), "w") as f:
        f.write(f"name {meta['name']}\n")
        f.write(f"digest {meta['digest']}\n")
        f.write(f"N {meta['N']}\nQ {meta['Q']}\nM {meta['M']}\nblock {block}\n")
        f.write("W " + " ".join(repr(w) for w in meta["W"]) + "\n")
    if os.path.exists(out):
        shutil.rmtree(out)
    os.replace(tmp, out)
    if verbose:
        print(f"built {out}: codegen {meta['codegen_s']}s nvcc {meta['nvcc_s']}s {meta['kernels']}")
    return out


def _parse_ptxas(log: str) -> dict:
    res = {}
    cur = None
    for line in log.splitlines():
        m = re.search(r"Compiling entry function '(\w+)'", line)
        if m:
            cur = m.group(1)
            res[cur] = {}
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            res[cur].update(stack=int(m.group(1)), spill_st=int(m.group(2)), spill_ld=int(m.group(3)))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            res[cur]["regs"] = int(m.group(1))
    return res


def load_meta(art_dir: str) -> dict:
    with open(os.path.join(art_dir, "meta.json")) as f:
        return json.load(f)
