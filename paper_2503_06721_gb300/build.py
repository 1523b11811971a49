"""Builds libhr.so (CUDA, sm_103a) in-tree from csrc/ with nvcc.

The hopping and represent/force kernels are templated on (N, representation);
each pair is compiled as its own translation unit so the build runs in
parallel.  Objects are cached by modification time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
OUTDIR = PKG / "_lib"
OBJDIR = PKG / "_build"
LIB = OUTDIR / "libhr.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              f"-I{INCLUDE}", f"-I{CSRC}"]

PRECS = ["HR_F64", "HR_F32", "HR_F16", "HR_BF16", "HR_DF64"]
PAIRS = [(2, "HR_FUND"), (2, "HR_ADJ"), (2, "HR_SYM"), (3, "HR_FUND"), (3, "HR_ADJ"), (3, "HR_SYM"),
         (3, "HR_ASYM"), (4, "HR_FUND"), (4, "HR_ASYM"), (4, "HR_ASYM_REAL")]
# pairs run by the colour-parallel hopping kernel (FP64 and FP32): the
# fundamental of large N and the SU(4) adjoint and symmetric representations
LARGE_PAIRS = [(5, "HR_FUND"), (6, "HR_FUND"), (8, "HR_FUND"), (4, "HR_ADJ"), (4, "HR_SYM")]


def _units():
    units = []
    for src in ("hr_api.cu", "hr_cg.cu", "hr_mscg.cu", "hr_hmc.cu", "hr_clover.cu", "hr_blas.cu", "hr_static.cu", "hr_tune.cu",
                "hr_rational.cu"):
        units.append((CSRC / src, OBJDIR / (Path(src).stem + ".o"), []))
    for n, rep in PAIRS:
        tag = f"{n}_{rep.lower()[3:]}"
        units.append((CSRC / "hr_gauge_inst.cu", OBJDIR / f"hr_gauge_inst_{tag}.o",
                      [f"-DHR_INST_N={n}", f"-DHR_INST_REP={rep}"]))
        for prec in PRECS:
            units.append((CSRC / "hr_dslash_inst.cu",
                          OBJDIR / f"hr_dslash_inst_{tag}_{prec.lower()[3:]}.o",
                          [f"-DHR_INST_N={n}", f"-DHR_INST_REP={rep}", f"-DHR_INST_P={prec}"]))
    for n, rep in LARGE_PAIRS:
        tag = f"{n}_{rep.lower()[3:]}"
        units.append((CSRC / "hr_gauge_inst.cu", OBJDIR / f"hr_gauge_inst_{tag}.o",
                      [f"-DHR_INST_N={n}", f"-DHR_INST_REP={rep}"]))
        for prec in ("HR_F64", "HR_F32"):
            units.append((CSRC / "hr_dslash_colour.cu", OBJDIR / f"hr_dslash_colour_{tag}_{prec.lower()[3:]}.o",
                          [f"-DHR_INST_N={n}", f"-DHR_INST_REP={rep}", f"-DHR_INST_P={prec}"]))
    return units


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> Path:
    OUTDIR.mkdir(exist_ok=True)
    OBJDIR.mkdir(exist_ok=True)
    headers = list(CSRC.glob("*.cuh")) + [INCLUDE / "hr.h"]
    hdr_time = max(h.stat().st_mtime for h in headers)
    nvcc = _nvcc()
    todo = []
    for src, obj, defs in _units():
        stale = force or not obj.exists() or obj.stat().st_mtime < max(hdr_time, src.stat().st_mtime)
        if stale:
            todo.append([nvcc, *NVCC_FLAGS, *ARCH, *defs, "-c", str(src), "-o", str(obj)])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return cmd[-1]

    jobs = jobs or max(1, os.cpu_count() or 1)
    # longest units first
    def weight(cmd):
        obj = cmd[-1]
        if "dslash" in obj:
            return 0 if obj.endswith(("_f32.o", "_f16.o", "_bf16.o")) else 1
        return 2
    todo.sort(key=weight)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for f in cf.as_completed([ex.submit(run, c) for c in todo]):
            f.result()
    objs = [str(o) for _, o, _ in _units()]
    if todo or not LIB.exists() or LIB.stat().st_mtime < max(Path(o).stat().st_mtime for o in objs):
        tmp = OUTDIR / f"libhr.{os.getpid()}.so"
        cmd = [nvcc, "-shared", *ARCH, "-o", str(tmp), *objs, "-lcudart_static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time
    t0 = time.time()
    p = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(p, f"{time.time() - t0:.1f}s")
