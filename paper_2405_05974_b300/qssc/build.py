"""Compile a mechanism into a loadable artefact (cubin + metadata).

    build_mechanism(mech_dict) -> artefact directory

The directory holds ``mech_body.inc`` (the generated code), ``mech.cubin``
(sm_103a: device math, the generated body and the wdot/Jacobian kernels),
``newton.cubin`` (the implicit-step kernels, which need only the mechanism's
sizes and molar masses), ``meta.txt`` (read by the C runtime) and
``meta.json`` (op counts, registers, spills).  Artefact directories are keyed
by the mechanism, the generator and the templates; each cubin is also cached
by the hash of its source, headers and flags under ``build/cubins``, so a
change to the Newton kernels does not recompile the generated body.
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
    for f in ("emit.py", "model.py", "expr.py", "mech.py", "graph.py"):
        h.update(open(os.path.join(os.path.dirname(__file__), f), "rb").read())
    return h.hexdigest()[:12]


def artefact_key(mech: dict, block: int = 128, defines=()) -> str:
    """Key of the artefact directory: the mechanism, the code generator and
    the hand-written templates (each cubin is also cached by content)."""
    h = hashlib.sha256(json.dumps(mech, sort_keys=True).encode())
    h.update(f"{block}|{sorted(defines)}|{_template_digest()}".encode())
    for t in TEMPLATES:
        p = os.path.join(CSRC, t)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:20]


CUBIN_CACHE = os.path.join(REPO, "build", "cubins")


def _compile_cubin(tu_src: str, headers: dict, flags, out_path: str, log_path: str):
    """Compile one translation unit to a cubin, cached by the hash of its
    source, the headers it includes (name -> text) and the flags."""
    h = hashlib.sha256(tu_src.encode())
    for name in sorted(headers):
        h.update(name.encode())
        h.update(headers[name].encode())
    h.update(" ".join(flags).encode())
    key = h.hexdigest()[:24]
    cached = os.path.join(CUBIN_CACHE, key + ".cubin")
    cached_log = os.path.join(CUBIN_CACHE, key + ".log")
    if not os.path.exists(cached):
        os.makedirs(CUBIN_CACHE, exist_ok=True)
        work = cached + ".d%d" % os.getpid()
        os.makedirs(work, exist_ok=True)
        for name, text in headers.items():
            if not os.path.exists(os.path.join(CSRC, name)):
                with open(os.path.join(work, name), "w") as f:
                    f.write(text)
        with open(os.path.join(work, "tu.cu"), "w") as f:
            f.write(tu_src)
        cmd = [NVCC, "-cubin", *ARCH, "-O3", "-lineinfo", "-Xptxas", "-v", *flags, "-I", CSRC,
               "-I", work, "-o", cached + ".tmp", os.path.join(work, "tu.cu")]
        p = subprocess.run(cmd, capture_output=True, text=True)
        log = " ".join(cmd) + "\n" + p.stdout + p.stderr
        shutil.rmtree(work, ignore_errors=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{log[-4000:]}")
        with open(cached_log, "w") as f:
            f.write(log)
        os.replace(cached + ".tmp", cached)
    shutil.copyfile(cached, out_path)
    shutil.copyfile(cached_log, log_path)
    return open(log_path).read()


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
    # sizes and constants only (for the Newton kernels' translation unit)
    sizes = src[:src.index("__device__ __forceinline__ void qss_eval_wdot")]
    hdr = {t: open(os.path.join(CSRC, t)).read() for t in TEMPLATES if os.path.exists(os.path.join(CSRC, t))}
    flags = [f"-DQSS_BLOCK={block}", *[f"-D{d}" for d in defines]]
    t1 = time.time()
    tu_mech = '#include "qss_device.cuh"\n#include "mech_body.inc"\n#include "qss_kernels.cuh"\n'
    common = {k: hdr[k] for k in ("qss_device.cuh", "qss_exp_table.inc")}
    log = _compile_cubin(tu_mech, {**common, "qss_kernels.cuh": hdr["qss_kernels.cuh"], "mech_body.inc": src},
                         flags, os.path.join(tmp, "mech.cubin"), os.path.join(tmp, "build.log"))
    t2 = time.time()
    tu_newton = '#include "qss_device.cuh"\n#include "mech_sizes.inc"\n#include "qss_newton.cuh"\n'
    log_n = _compile_cubin(tu_newton, {**common, "qss_newton.cuh": hdr["qss_newton.cuh"],
                                       "mech_sizes.inc": sizes}, flags,
                           os.path.join(tmp, "newton.cubin"), os.path.join(tmp, "build_newton.log"))
    meta["kernels"] = {**_parse_ptxas(log), **_parse_ptxas(log_n)}
    meta["block"] = block
    meta["defines"] = list(defines)
    meta["codegen_s"] = round(t1 - t0, 3)
    meta["nvcc_s"] = round(t2 - t1, 3)
    meta["nvcc_newton_s"] = round(time.time() - t2, 3)
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
        print(f"built {out}: codegen {meta['codegen_s']}s nvcc {meta['nvcc_s']}s + {meta['nvcc_newton_s']}s "
              f"{meta['kernels']}")
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
