"""Build libaderdg.so in-tree for sm_103a with nvcc.

The kernel templates are instantiated per (PDE, d, N, precision, predictor)
in generated translation units, compiled in parallel, and linked with the
host orchestration into ``_build/libaderdg.so``.  Each unit registers its
configurations when the library is loaded.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libaderdg.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-v", "-I", INCLUDE, "-I", CSRC] + ARCH

PDE_T = {"advection": ("Advection", 0), "acoustics": ("Acoustics", 1),
         "euler": ("Euler", 2), "elasticity": ("Elasticity", 3)}
PREC_T = {"fp32": ("float", "float", 0), "fp64": ("double", "double", 1),
          "acc64": ("float", "double", 2), "pair": ("float", "Pair32", 3)}
PRED_T = {"tm": "kTimeModal", "st": "kSpaceTime", "tc": "kSpaceTimeTC"}


def configs():
    """(pde, d, N, precision, predictor, with_table1, with_adjoint, with_ext) compiled into the
    library; with_ext adds the fused-sweep kernels with point sources and material jumps in
    non-conservative form."""
    out = []

    def add(pde, ds, Ns, precs, preds, t1=(), adj=(), ext=()):
        for d in ds:
            for N in Ns:
                for p in precs:
                    for pr in preds:
                        key = (d, N, p, pr)
                        out.append((pde, d, N, p, pr, key in t1, key in adj, key in ext))

    # linear advection: 2D workload in FP64, FV case N=0, small 3D cases
    add("advection", [2], range(0, 7), ["fp32", "fp64"], ["tm"],
        ext={(2, N, "fp64", "tm") for N in (1, 2, 3)})
    add("advection", [3], range(1, 4), ["fp32"], ["tm"])
    add("advection", [2], [1, 3], ["fp64"], ["st"], t1={(2, 3, "fp64", "st")})
    # linear acoustics: the 3D N=5 workload, the 2D ensemble orders
    add("acoustics", [2], range(0, 7), ["fp32"], ["tm"], t1={(2, 2, "fp32", "tm")},
        adj={(2, 2, "fp32", "tm")}, ext={(2, 3, "fp32", "tm")})
    add("acoustics", [3], range(1, 7), ["fp32"], ["tm"], t1={(3, 5, "fp32", "tm")},
        ext={(3, 3, "fp32", "tm")})
    add("acoustics", [2, 3], [1, 2, 3], ["fp64"], ["tm"], t1={(2, 2, "fp64", "tm")},
        adj={(2, 2, "fp64", "tm")}, ext={(2, 3, "fp64", "tm")})
    add("acoustics", [2], [0], ["fp64"], ["tm"])
    add("acoustics", [3], [5], ["fp32"], ["st"], t1={(3, 5, "fp32", "st")})
    add("acoustics", [2], [2], ["fp64"], ["st"])
    # compressible Euler: space-time Picard only
    add("euler", [2], range(0, 5), ["fp32", "fp64"], ["st"], t1={(2, 2, "fp64", "st")})
    add("euler", [2], [2, 3], ["acc64"], ["st"])
    add("euler", [3], [2, 3, 4], ["fp32", "acc64"], ["st"], t1={(3, 3, "fp32", "st")})
    add("euler", [3], [2], ["fp64"], ["st"])
    # space-time Picard with tensor-core (TF32) flux-divergence contractions
    add("euler", [2], [2, 3], ["fp32"], ["tc"])
    add("euler", [3], [2, 3], ["fp32", "acc64"], ["tc"])
    add("acoustics", [3], [3], ["fp32"], ["tc"])
    # elasticity: the 3D N=4 workload, the 2D ensemble orders
    add("elasticity", [2], range(0, 7), ["fp32"], ["tm"], adj={(2, 2, "fp32", "tm"), (2, 3, "fp32", "tm")},
        ext={(2, 3, "fp32", "tm")})
    add("elasticity", [3], range(2, 6), ["fp32"], ["tm"], t1={(3, 4, "fp32", "tm")},
        adj={(3, 2, "fp32", "tm"), (3, 4, "fp32", "tm")}, ext={(3, 4, "fp32", "tm")})
    add("elasticity", [2, 3], [2], ["fp64"], ["tm"], adj={(2, 2, "fp64", "tm"), (3, 2, "fp64", "tm")},
        ext={(2, 2, "fp64", "tm"), (3, 2, "fp64", "tm")})
    add("elasticity", [2], [3], ["fp64"], ["tm"], ext={(2, 3, "fp64", "tm")})
    # compensated FP32 pair (and FP64) accumulation of the state: the three 3D
    # workloads and small cases for the tests
    add("acoustics", [3], [5], ["pair", "acc64"], ["tm"])
    add("acoustics", [2, 3], [2, 3], ["pair", "acc64"], ["tm"])
    add("elasticity", [3], [4], ["pair"], ["tm"])
    add("elasticity", [2], [3], ["pair"], ["tm"])
    add("euler", [3], [3], ["pair"], ["st"])
    add("euler", [2], [2, 3], ["pair"], ["st"])
    return out


def unit_source(group):
    lines = ['#include "kernels.cuh"', "namespace aderdg {", "namespace {"]
    for i, (pde, d, N, prec, pred, t1, adj, ext) in enumerate(group):
        tname, pid = PDE_T[pde]
        R, QT, precid = PREC_T[prec]
        K = f"Cfg<{tname}, {d}, {N}, {R}, {QT}, {PRED_T[pred]}>"
        flags = f"{'true' if t1 else 'false'}, {'true' if adj else 'false'}, {'true' if ext else 'false'}"
        lines.append(f"Registrar r{i}(make_set<{K}, {flags}>({pid}, {precid}));")
    lines += ["}  // namespace", "}  // namespace aderdg", ""]
    return "\n".join(lines)


def groups(per_unit=3):
    cfg = configs()
    return [cfg[i:i + per_unit] for i in range(0, len(cfg), per_unit)]


def _hash_inputs():
    h = hashlib.sha1()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    with open(os.path.join(INCLUDE, "aderdg.h"), "rb") as f:
        h.update(f.read())
    h.update(repr(configs()).encode())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed: {' '.join(cmd)}\n{r.stdout}")
    return r.stdout


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every unit (parallel) and link the shared library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    key = _hash_inputs()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == key:
        return LIB
    gen = os.path.join(BUILD, "gen")
    os.makedirs(gen, exist_ok=True)
    units = []
    for name in ("api.cu", "noalloc.cu", "batch.cu", "peak.cu", "basis.cpp"):
        units.append(os.path.join(CSRC, name))
    for i, grp in enumerate(groups()):
        path = os.path.join(gen, f"inst_{i:03d}.cu")
        src = unit_source(grp)
        if not os.path.exists(path) or open(path).read() != src:
            with open(path, "w") as f:
                f.write(src)
        units.append(path)
    objs = []
    cmds = []
    for u in units:
        o = os.path.join(BUILD, os.path.basename(u) + ".o")
        objs.append(o)
        if u.endswith(".cpp"):
            cmds.append(["g++", "-std=c++17", "-O2", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-c", u, "-o", o])
        else:
            cmds.append(["nvcc"] + NVCC_FLAGS + ["-c", u, "-o", o])
    jobs = jobs or max(1, os.cpu_count() or 1)
    with ThreadPoolExecutor(jobs) as ex:
        outs = list(ex.map(_run, cmds))
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        f.write("\n".join(outs))
    if verbose:
        print("\n".join(o for o in outs if o.strip()))
    tmp = LIB + f".{os.getpid()}.tmp"
    _run(["nvcc", "-shared"] + ARCH + ["-o", tmp] + objs)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(key)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
