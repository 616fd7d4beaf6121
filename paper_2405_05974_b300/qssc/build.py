"""Compile a mechanism into a loadable artefact (cubin + metadata).

    build_mechanism(mech_dict) -> artefact directory

The directory holds the generated code (``mech_sizes.inc``: sizes and
constants; ``mech_wdot.inc``: the source term; ``mech_jac.inc``: the
Jacobian), three sm_103a cubins compiled in parallel from three translation
units -- ``jac.cubin`` (the analytic Jacobian kernel), ``wdot.cubin`` (the
source-term and finite-difference Jacobian kernels) and ``newton.cubin`` (the
implicit-step kernels, which need only the sizes and molar masses) --
``meta.txt`` (read by the C runtime) and ``meta.json`` (op counts, registers,
spills).  Artefact directories are keyed by the mechanism, the generator, the
options and the templates; each cubin is also cached by the hash of its
source, headers and flags under ``build/cubins``, so a change to one kernel
template does not recompile the others' generated code.
"""
from __future__ import annotations

import hashlib
import json
import os
import re
import shutil
import subprocess
import threading
import time
from concurrent.futures import ThreadPoolExecutor

from . import emit, mech as qmech, model as qmodel

PKG = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(PKG, "csrc")
REPO = os.path.dirname(PKG)
DEFAULT_ROOT = os.path.join(REPO, "build", "mech")
NVCC = os.environ.get("QSS_NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
TEMPLATES = ["qss_device.cuh", "qss_exp_table.inc", "qss_log_table.inc", "qss_cells.cuh",
             "qss_jac_kernel.cuh", "qss_jac_parts.cuh", "qss_wdot_kernels.cuh", "qss_newton.cuh",
             "qss_convert.h", "qss_jac32_kernel.cuh", "qss_jac2_kernel.cuh"]
ARTEFACT_FILES = ("meta.txt", "meta.json")   # plus the cubins meta.txt names
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
# Artefacts of one mechanism share most of their cubins (the source-term and
# Newton cubins do not depend on the Jacobian's build options, and variants
# differ in one kernel), so each distinct cubin is stored once, in this
# directory beside the artefact directories, named by its content key;
# meta.txt maps the artefact's cubin names to it ("cubin wdot.cubin
# ../_cubins/<key>.cubin").
SHARED = "_cubins"


def cubin_file(art: str, name: str) -> str:
    """Path of the artefact's cubin `name` ("jac.cubin", "wdot.cubin", ...)."""
    rel = _cubin_map(art).get(name)
    return os.path.normpath(os.path.join(art, rel)) if rel else os.path.join(art, name)


def source_dir(art: str) -> str:
    """Directory of the generated sources (mech_*.inc) of artefact `art`."""
    art = os.path.normpath(art)
    return os.path.join(os.path.dirname(os.path.dirname(art)), "src", os.path.basename(art))


def _cubin_map(art: str) -> dict:
    out = {}
    try:
        with open(os.path.join(art, "meta.txt")) as f:
            for ln in f:
                p = ln.split()
                if len(p) == 3 and p[0] == "cubin":
                    out[p[1]] = p[2]
    except OSError:
        pass
    return out


def _compile_cubin(tu_src: str, headers: dict, flags, store: str, log_path: str):
    """Compile one translation unit to a cubin, cached by the hash of its
    source, the headers it includes (name -> text) and the flags; the cubin
    is placed in the shared store `store` under its key.  Returns (ptxas
    log, key)."""
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
        tag = "%d_%d" % (os.getpid(), threading.get_ident())
        work = cached + ".d" + tag
        os.makedirs(work, exist_ok=True)
        for name, text in headers.items():
            if not os.path.exists(os.path.join(CSRC, name)):
                with open(os.path.join(work, name), "w") as f:
                    f.write(text)
        with open(os.path.join(work, "tu.cu"), "w") as f:
            f.write(tu_src)
        cmd = [NVCC, "-cubin", *ARCH, "-O3", "-lineinfo", "-Xptxas", "-v", *flags, "-I", CSRC,
               "-I", work, "-o", cached + ".tmp" + tag, os.path.join(work, "tu.cu")]
        p = subprocess.run(cmd, capture_output=True, text=True)
        log = " ".join(cmd) + "\n" + p.stdout + p.stderr
        shutil.rmtree(work, ignore_errors=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{log[-4000:]}")
        with open(cached_log, "w") as f:
            f.write(log)
        os.replace(cached + ".tmp" + tag, cached)
    dst = os.path.join(store, key + ".cubin")
    if not os.path.exists(dst):
        os.makedirs(store, exist_ok=True)
        tmp = dst + ".tmp%d_%d" % (os.getpid(), threading.get_ident())
        shutil.copyfile(cached, tmp)
        os.replace(tmp, dst)
    shutil.copyfile(cached_log, log_path)
    return open(log_path).read(), key


_INDEX_LOCK = threading.Lock()


def _read_index(root: str) -> dict:
    try:
        with open(os.path.join(root, "index.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _write_index(root: str, fast: str, name: str):
    """Record fast key -> artefact directory (read-modify-write under a lock;
    concurrent processes at worst lose an entry, which costs one codegen)."""
    with _INDEX_LOCK:
        idx = _read_index(root)
        if idx.get(fast) == name:
            return
        idx[fast] = name
        os.makedirs(root, exist_ok=True)
        tmp = os.path.join(root, "index.json.tmp%d_%d" % (os.getpid(), threading.get_ident()))
        with open(tmp, "w") as f:
            json.dump(idx, f, indent=0, sort_keys=True)
        os.replace(tmp, os.path.join(root, "index.json"))


def _variant(jac_variant, t_column, jac_parts, replace_nop, jac_format, emit_order, smem_slots, ptxas,
             jac32=False, jac32_slots=0, jac32_minblocks=1, cells_per_thread=1) -> tuple:
    """The build options other than block and defines, as index-key parts."""
    variant = () if (jac_variant, t_column) == ("exact", "analytic") else (f"{jac_variant}/{t_column}",)
    if jac_parts >= 2:
        variant += (f"parts{int(jac_parts)}",)
    if replace_nop > 0:
        variant += (f"nop{int(replace_nop)}",)
    if jac_format != "dense":
        variant += (jac_format,)
    if emit_order != "first_use":
        variant += (emit_order,)
    if smem_slots > 0:
        variant += (f"smem{int(smem_slots)}",)
    for o in ptxas:
        variant += (f"ptxas:{o}",)
    if jac32:
        if replace_nop > 0 or (jac_variant, t_column) != ("exact", "analytic"):
            raise ValueError("jac32 is built for the exact Jacobian with the analytic T column")
        variant += ("jac32",)
    if jac32_slots > 0:
        if not jac32 or jac_parts >= 2:
            raise ValueError("jac32_slots applies to the single-kernel mixed-precision Jacobian")
        variant += (f"j32smem{int(jac32_slots)}",)
    if jac32_minblocks != 1:
        if not jac32 or jac_parts >= 2:
            raise ValueError("jac32_minblocks applies to the single-kernel mixed-precision Jacobian")
        variant += (f"j32mb{int(jac32_minblocks)}",)
    if cells_per_thread != 1:
        if cells_per_thread != 2 or jac_parts >= 2 or smem_slots > 0 or t_column != "analytic":
            raise ValueError("cells_per_thread = 2 applies to the single FP64 Jacobian kernel without "
                             "shared-memory values, analytic temperature column")
        variant += ("cpt2",)
    return variant


def find_artefact(mech: dict, root: str = None, block: int = 128, defines=(), jac_variant: str = "exact",
                  t_column: str = "analytic", jac_parts: int = 0, replace_nop: int = 0,
                  jac_format: str = "dense", emit_order: str = "first_use", smem_slots: int = 0, ptxas=(),
                  jac32: bool = False, jac32_slots: int = 0, jac32_minblocks: int = 1, cells_per_thread: int = 1):
    """The directory of an artefact already built with these options for the
    current templates, or None (never compiles)."""
    root = root or DEFAULT_ROOT
    variant = _variant(jac_variant, t_column, jac_parts, replace_nop, jac_format, emit_order, smem_slots, ptxas,
                       jac32, jac32_slots, jac32_minblocks, cells_per_thread)
    name = _read_index(root).get(artefact_key(mech, block, tuple(defines) + variant))
    return os.path.join(root, name) if name and _complete(os.path.join(root, name)) else None


def prune_artefacts(keep, root: str = None) -> list:
    """Remove the artefact directories under `root` that are not in `keep`
    (paths returned by build_mechanism in this build) and their index
    entries: a template or generator change leaves the previous artefacts
    behind, and the tree would otherwise grow with every such change.
    Returns the removed directory names."""
    root = root or DEFAULT_ROOT
    keep_names = {os.path.basename(os.path.normpath(k)) for k in keep}
    removed = []
    with _INDEX_LOCK:
        idx = {k: v for k, v in _read_index(root).items() if v in keep_names}
        tmp = os.path.join(root, "index.json.tmp%d" % os.getpid())
        with open(tmp, "w") as f:
            json.dump(idx, f, indent=0, sort_keys=True)
        os.replace(tmp, os.path.join(root, "index.json"))
        for d in sorted(os.listdir(root)):
            p = os.path.join(root, d)
            # a ".tmp" directory younger than a day belongs to a build still
            # running in another process
            if ".tmp" in d and time.time() - os.path.getmtime(p) < 86400:
                continue
            if os.path.isdir(p) and d not in keep_names and d != SHARED:
                shutil.rmtree(p, ignore_errors=True)
                removed.append(d)
        srcroot = os.path.join(os.path.dirname(os.path.normpath(root)), "src")
        for d in sorted(os.listdir(srcroot)) if os.path.isdir(srcroot) else []:
            if d not in keep_names:
                shutil.rmtree(os.path.join(srcroot, d), ignore_errors=True)
        # shared cubins no kept artefact refers to
        used = {os.path.basename(r) for k in keep_names for r in _cubin_map(os.path.join(root, k)).values()}
        store = os.path.join(root, SHARED)
        for f in sorted(os.listdir(store)) if os.path.isdir(store) else []:
            if f not in used:
                os.remove(os.path.join(store, f))
    return removed


def _complete(out: str) -> bool:
    if not all(os.path.exists(os.path.join(out, f)) for f in ("meta.txt", "meta.json")):
        return False
    m = _cubin_map(out)
    if not m:
        return False
    have = lambda f: f in m and os.path.exists(os.path.normpath(os.path.join(out, m[f])))  # noqa: E731
    return all(have(f) for f in m) and have("wdot.cubin") and have("newton.cubin") and (
        have("jac.cubin") or have("jac_prefix.cubin"))


def build_mechanism(mech: dict, root: str = DEFAULT_ROOT, block: int = 128, defines=(),
                    force: bool = False, verbose: bool = False, jac_variant: str = "exact",
                    t_column: str = "analytic", jac_parts: int = 0, replace_nop: int = 0,
                    jac_format: str = "dense", emit_order: str = "first_use", smem_slots: int = 0,
                    ptxas=(), jac32: bool = False, jac32_slots: int = 0, jac32_minblocks: int = 1,
                    cells_per_thread: int = 1) -> str:
    """Generate, compile and cache the artefact of one mechanism.

    ``jac_variant`` / ``t_column`` select the Jacobian that the kernels
    compute (``model.build_model``); ``defines`` are extra preprocessor
    definitions of the kernel templates (e.g. ``QSS_MINBLOCKS=2``);
    ``jac_parts`` >= 2 splits the Jacobian into a prefix kernel and that many
    column-group kernels (``emit.emit_partitioned_source``), each compiled in
    its own translation unit; ``replace_nop`` > 0 applies Alg. 2's
    common-subexpression replacement with that operation threshold;
    ``jac_format`` "csr" makes the Jacobian kernels store only the structural
    nonzeros, in CSR order (``emit.jac_layout``); ``emit_order`` "all_first"
    computes every value before any output is stored (Alg. 3's recycling off,
    for the memory study; the default "first_use" stores each output as soon
    as it is final); ``smem_slots`` > 0 keeps that many of the FP64 Jacobian
    kernel's most-reloaded values in shared memory (dynamic, per thread; with
    ``jac_parts`` in the prefix and in each column-group kernel);
    ``cells_per_thread`` = 2 makes each thread of the FP64 Jacobian kernel
    evaluate two cells (the body and its copy interleaved,
    ``emit.two_cell_body``, in the kernel of qss_jac2_kernel.cuh);
    ``ptxas`` are extra ptxas options (``"regUsageLevel=0"`` is passed as
    ``-Xptxas -regUsageLevel=0``); ``jac32`` also builds ``jac32.cubin``, the
    mixed-precision Jacobian kernel (derivative terms in FP32,
    ``emit.emit_jac32_source``) of the mixed-precision implicit step, with
    ``jac32_slots`` of its most-reloaded FP32 values in shared memory and
    ``jac32_minblocks`` blocks per SM in its register budget (its own
    __launch_bounds__, so the other cubins are unaffected)."""
    variant = _variant(jac_variant, t_column, jac_parts, replace_nop, jac_format, emit_order, smem_slots, ptxas,
                       jac32, jac32_slots, jac32_minblocks, cells_per_thread)
    # fast path: the key of (mechanism, options, generator, templates) in the
    # index of built artefacts
    fast = artefact_key(mech, block, tuple(defines) + variant)
    index = _read_index(root)
    if not force and fast in index and _complete(os.path.join(root, index[fast])):
        return os.path.join(root, index[fast])
    t0 = time.time()
    ir = qmech.parse(mech)
    model = qmodel.build_model(ir, jac_variant=jac_variant, t_column=t_column)
    src, meta = emit.emit_mechanism_source(model, replace_nop=replace_nop, jac_format=jac_format,
                                           emit_order=emit_order,
                                           smem_slots=smem_slots if jac_parts < 2 else 0,
                                           cells_per_thread=cells_per_thread)
    # sizes and constants / the source term / the Jacobian, one file each
    iw = src.index("__device__ __forceinline__ void qss_eval_wdot")
    ij = src.index("__device__ __forceinline__ void qss_eval_jac")
    parts = {"mech_sizes.inc": src[:iw], "mech_wdot.inc": src[iw:ij], "mech_jac.inc": src[ij:]}
    if jac_parts >= 2:
        prefix_src, group_srcs, pmeta = emit.emit_partitioned_source(model, int(jac_parts), jac_format,
                                                                     smem_slots=smem_slots)
        meta.update(pmeta)
        # every kernel of the partition is launched with the largest count
        meta["smem_slots"] = max(pmeta["smem_slots_parts"])
        del parts["mech_jac.inc"]
        parts["mech_jac_prefix.inc"] = prefix_src
        for i, gsrc in enumerate(group_srcs):
            parts[f"mech_jac_g{i}.inc"] = gsrc
    if jac32 and jac_parts < 2:
        src32, meta32 = emit.emit_jac32_source(model, jac_format, smem_slots=jac32_slots)
        parts["mech_jac32.inc"] = src32
        meta.update(meta32)
    elif jac32:
        p32, g32, pm32 = emit.emit_partitioned_source(model, int(jac_parts), jac_format, mixed=True)
        parts["mech_jac32_prefix.inc"] = p32
        for i, gsrc in enumerate(g32):
            parts[f"mech_jac32_g{i}.inc"] = gsrc
        meta.update({"ops_prefix32": pm32["ops_prefix"], "ops_groups32": pm32["ops_groups"]})
    hdr = {t: open(os.path.join(CSRC, t)).read() for t in TEMPLATES}
    flags = [f"-DQSS_BLOCK={block}", *[f"-D{d}" for d in defines]]
    for o in ptxas:
        flags += ["-Xptxas", f"-{o}"]
    # the directory is keyed by what is compiled: the generated sources, the
    # templates and the flags (a generator change that emits the same code
    # keeps its artefacts)
    hk = hashlib.sha256(json.dumps([sorted(parts.items()), sorted(hdr.items()), flags,
                                    meta.get("jac_variant"), meta.get("t_column"), jac_parts]
                                   + ([jac32_minblocks] if jac32_minblocks != 1 else [])
                                   + (["cpt2"] if cells_per_thread == 2 else [])).encode())
    art_name = f"{mech.get('name', 'mech')}_{hk.hexdigest()[:20]}"
    out = os.path.join(root, art_name)
    if not force and _complete(out):
        _write_index(root, fast, art_name)
        return out
    tmp = out + ".tmp%d_%d" % (os.getpid(), threading.get_ident())   # one per concurrent build
    os.makedirs(tmp, exist_ok=True)
    # the generated sources (inputs of the compile, not needed to load the
    # artefact) are kept beside the artefacts, not in them
    srcd = source_dir(out)
    os.makedirs(srcd, exist_ok=True)
    for pname, text in parts.items():
        with open(os.path.join(srcd, pname), "w") as f:
            f.write(text)
    t1 = time.time()
    common = {k: hdr[k] for k in ("qss_device.cuh", "qss_exp_table.inc", "qss_log_table.inc")}
    cells = {"qss_cells.cuh": hdr["qss_cells.cuh"], "mech_sizes.inc": parts["mech_sizes.inc"]}
    pre = '#include "qss_device.cuh"\n#include "mech_sizes.inc"\n'
    units = {}
    if jac_parts >= 2:
        jp = {"qss_jac_parts.cuh": hdr["qss_jac_parts.cuh"]}
        units["jac_prefix"] = (pre + '#include "mech_jac_prefix.inc"\n#define QSS_JAC_PREFIX\n'
                               '#include "qss_jac_parts.cuh"\n',
                               {**common, **cells, **jp, "mech_jac_prefix.inc": parts["mech_jac_prefix.inc"]})
        for i in range(int(jac_parts)):
            nm = f"mech_jac_g{i}.inc"
            units[f"jac_g{i}"] = (pre + f'#include "{nm}"\n#define QSS_JAC_GROUP\n#include "qss_jac_parts.cuh"\n',
                                  {**common, **cells, **jp, nm: parts[nm]})
    else:
        kt = "qss_jac2_kernel.cuh" if cells_per_thread == 2 else "qss_jac_kernel.cuh"
        units["jac"] = (pre + f'#include "mech_jac.inc"\n#include "{kt}"\n',
                        {**common, **cells, "mech_jac.inc": parts["mech_jac.inc"], kt: hdr[kt]})
    if jac32 and jac_parts >= 2:
        jp = {"qss_jac_parts.cuh": hdr["qss_jac_parts.cuh"], "qss_convert.h": hdr["qss_convert.h"]}
        cv = '#include "qss_convert.h"\n'
        units["jac32_prefix"] = (pre + cv + '#include "mech_jac32_prefix.inc"\n#define QSS_JAC_PREFIX\n'
                                 '#include "qss_jac_parts.cuh"\n',
                                 {**common, **cells, **jp, "mech_jac32_prefix.inc": parts["mech_jac32_prefix.inc"]})
        for i in range(int(jac_parts)):
            nm = f"mech_jac32_g{i}.inc"
            units[f"jac32_g{i}"] = (pre + cv + f'#include "{nm}"\n#define QSS_JAC_GROUP\n#include "qss_jac_parts.cuh"\n',
                                    {**common, **cells, **jp, nm: parts[nm]})
    elif jac32:
        units["jac32"] = (pre + '#include "qss_convert.h"\n#include "mech_jac32.inc"\n#include "qss_jac32_kernel.cuh"\n',
                          {**common, **cells, "qss_convert.h": hdr["qss_convert.h"],
                           "mech_jac32.inc": parts["mech_jac32.inc"],
                           "qss_jac32_kernel.cuh": hdr["qss_jac32_kernel.cuh"]})
    units.update({
        "wdot": (pre + '#include "mech_wdot.inc"\n#include "qss_wdot_kernels.cuh"\n',
                 {**common, **cells, "mech_wdot.inc": parts["mech_wdot.inc"],
                  "qss_wdot_kernels.cuh": hdr["qss_wdot_kernels.cuh"]}),
        "newton": (pre + '#include "qss_newton.cuh"\n',
                   {**common, "mech_sizes.inc": parts["mech_sizes.inc"],
                    "qss_newton.cuh": hdr["qss_newton.cuh"]}),
    })
    logs, secs, keys = {}, {}, {}

    def compile_unit(name):
        t = time.time()
        tu, headers = units[name]
        uflags = flags + ([f"-DQSS_J32_MINBLOCKS={int(jac32_minblocks)}"] if name == "jac32" and jac32_minblocks != 1
                          else [])
        logs[name], keys[name] = _compile_cubin(tu, headers, uflags, os.path.join(root, SHARED),
                                                os.path.join(tmp, f"build_{name}.log"))
        secs[name] = round(time.time() - t, 3)

    with ThreadPoolExecutor(min(len(units), os.cpu_count() or 4)) as ex:
        for f in [ex.submit(compile_unit, u) for u in units]:
            f.result()
    meta["kernels"] = {}
    for name in units:
        for k, v in _parse_ptxas(logs[name]).items():
            if name.startswith("jac_g"):
                k = f"{k}[{name[5:]}]"
            elif name.startswith("jac32_"):
                k = f"{k}[{name}]"
            meta["kernels"][k] = v
    meta["block"] = block
    meta["defines"] = list(defines)
    meta["ptxas"] = list(ptxas)
    meta["codegen_s"] = round(t1 - t0, 3)
    meta["nvcc_s"] = secs
    meta["artefact_key"] = art_name.rsplit("_", 1)[1]
    with open(os.path.join(tmp, "meta.json"), "w") as f:
        json.dump(meta, f, indent=1)
    with open(os.path.join(tmp, "meta.txt"), "w") as f:
        f.write(f"name {meta['name']}\n")
        f.write(f"digest {meta['digest']}\n")
        f.write(f"N {meta['N']}\nQ {meta['Q']}\nM {meta['M']}\nblock {block}\n")
        if jac_parts >= 2:
            f.write(f"jac_parts {int(jac_parts)}\nfrontier {meta['frontier']}\n")
        f.write(f"jac_nnz {meta['jac_stored']}\n")
        if jac32:
            f.write("jac32 1\n")
        if cells_per_thread == 2:
            f.write("cpt 2\n")
        if meta.get("jac32_slots", 0) > 0:
            f.write(f"jac32_slots {int(meta['jac32_slots'])}\n")
        if meta.get("smem_slots", 0) > 0:   # slots the emitted code uses (at most the requested)
            f.write(f"smem_slots {int(meta['smem_slots'])}\n")
        if jac_format != "dense":
            f.write("jac_row_ptr " + " ".join(map(str, meta["jac_row_ptr"])) + "\n")
            f.write("jac_col " + " ".join(map(str, meta["jac_col"])) + "\n")
        f.write("W " + " ".join(repr(w) for w in meta["W"]) + "\n")
        for name in sorted(units):
            f.write(f"cubin {name}.cubin ../{SHARED}/{keys[name]}.cubin\n")
    if os.path.exists(out):
        shutil.rmtree(out)
    os.replace(tmp, out)
    _write_index(root, fast, art_name)
    if verbose:
        print(f"built {out}: codegen {meta['codegen_s']}s nvcc {secs} {meta['kernels']}")
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
