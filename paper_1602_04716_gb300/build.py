"""Builds libbsfp.so (the CUDA library) in-tree for sm_103a.

Every translation unit compiles in parallel with one ``-gencode`` (sm_103a);
the element-wise kernels are split by exponent width and fraction range so
the instantiations spread over the cores.  Objects go to ``_build/`` next to
this file and are rebuilt only when a source or header is newer.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbsfp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
GEN_DIR = os.path.join(BUILD, "gen")
GEN_HEADER = os.path.join(GEN_DIR, "gen_circuits.cuh")
# Formats whose circuits are printed gate by gate from their netlists
# (circuitgen): the formats of the benchmarks and of the batched kernels.
GEN_FORMATS = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7), (8, 23)]
# Formats with a streamed kernel (stream.cuh): the generated formats of at
# most 16 planes.
STREAM_FORMATS = [(4, 3), (4, 4), (5, 7), (5, 10), (8, 7)]
# The element-wise kernels are compiled in parts: exponent width E and a
# range of fraction widths.  For every other format of a part, circuitgen
# prints add and mul under RN and RZ into that part's own header
# (gen_e<E>_m<lo>.cuh), which only the part's translation unit includes.
M_RANGES = ((1, 11), (12, 23))


def part_formats(e, lo, hi):
    return [(e, m) for m in range(lo, hi + 1) if 1 + e + m <= 32 and (e, m) not in GEN_FORMATS]


def part_header(e, lo):
    return "gen_e%d_m%d.cuh" % (e, lo)


def div_header(e, lo):
    """div (RN, RZ) of the part's other formats, printed for its division unit"""
    return "gen_div_e%d_m%d.cuh" % (e, lo)


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _units():
    """(object name, compiler command without -o) for every translation unit."""
    nv = nvcc()
    cu = [nv, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INC, "-I", GEN_DIR,
          "-DBSFP_HAVE_GEN", "-c"]
    units = []
    for e in range(2, 9):
        for lo, hi in M_RANGES:
            units.append(("binop_e%d_m%d.o" % (e, lo),
                          cu + ["-DBSFP_E=%d" % e, "-DBSFP_M_LO=%d" % lo, "-DBSFP_M_HI=%d" % hi, "-DBSFP_NO_DIV",
                                '-DBSFP_GEN_PART="%s"' % part_header(e, lo),
                                os.path.join(CSRC, "binop_inst.cu")]))
            units.append(("binop_div_e%d_m%d.o" % (e, lo),
                          cu + ["-DBSFP_E=%d" % e, "-DBSFP_M_LO=%d" % lo, "-DBSFP_M_HI=%d" % hi, "-DBSFP_DIV_UNIT",
                                '-DBSFP_GEN_PART="%s"' % div_header(e, lo),
                                os.path.join(CSRC, "binop_inst.cu")]))
        units.append(("gatecount_e%d.o" % e,
                      ["g++", "-std=c++17", "-O1", "-fPIC", "-I", CSRC, "-DBSFP_E=%d" % e, "-c",
                       os.path.join(CSRC, "gatecount.cpp")]))
        units.append(("conv_e%d.o" % e, cu + ["-DBSFP_E=%d" % e, os.path.join(CSRC, "conv_inst.cu")]))
    for lo, hi in ((1, 16), (17, 32)):
        units.append(("int_w%d.o" % lo, cu + ["-DBSFP_W_LO=%d" % lo, "-DBSFP_W_HI=%d" % hi,
                                               os.path.join(CSRC, "int_ops.cu")]))
    for e, m in STREAM_FORMATS:
        units.append(("stream_e%d_m%d.o" % (e, m), cu + ["-DBSFP_SE=%d" % e, "-DBSFP_SM=%d" % m,
                                                         os.path.join(CSRC, "stream_inst.cu")]))
    for e in range(2, 9):
        # streamed mul, fma2 and division of the other formats, each with the printed netlists of
        # this exponent width's formats (both parts)
        for op, opc, hdr in (("mul", 1, "gen_e%d_all.cuh"), ("fma2", 2, "gen_e%d_all.cuh"),
                             ("div", 3, "gen_div_e%d_all.cuh")):
            units.append(("stream_%s_e%d.o" % (op, e),
                          cu + ["-DBSFP_SE=%d" % e, "-DBSFP_SOPC=%d" % opc, "-DBSFP_GEN_PART=\"%s\"" % (hdr % e),
                                os.path.join(CSRC, "stream_band_inst.cu")]))
    for opc in range(3):
        units.append(("batch_opc%d.o" % opc, cu + ["-DBSFP_BATCH_OPC=%d" % opc, os.path.join(CSRC, "batch_inst.cu")]))
    for opc in range(2):
        units.append(("ustream_opc%d.o" % opc, cu + ["-DBSFP_USTREAM_OPC=%d" % opc,
                                                     os.path.join(CSRC, "ustream_inst.cu")]))
    for src in ("api.cu", "batch.cu", "batch_noalloc.cu", "serve.cu", "pipeline.cu", "autotune.cu", "transpose.cu", "probe.cu", "synth_gen.cu"):
        units.append((src.replace(".cu", ".o"), cu + [os.path.join(CSRC, src)]))
    return units


def _deps():
    return glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INC, "*.h"))


def _generate_one(defines, out_path, tag):
    """Compile circuitgen with the given format lists and print one header."""
    tool = os.path.join(BUILD, "circuitgen_" + tag)
    subprocess.check_call(["g++", "-std=c++17", "-O0", "-w", "-I", CSRC, *defines, os.path.join(CSRC, "circuitgen.cpp"),
                           "-o", tool])
    tmp = out_path + ".tmp"
    subprocess.check_call([tool, tmp])
    os.replace(tmp, out_path)


def generate(jobs: int | None = None) -> str:
    """Print the netlists: all ops and modes of GEN_FORMATS into
    _build/gen/gen_circuits.cuh, and add/mul (RN, RZ) of every other format
    into its part's header; redone only when a circuit source changed."""
    os.makedirs(GEN_DIR, exist_ok=True)
    srcs = [os.path.join(CSRC, f) for f in ("circuitgen.cpp", "netlist.h", "circuit.cuh")] + [__file__]
    newest = max(os.path.getmtime(p) for p in srcs)
    todo = []
    fmts = " ".join("X(%d, %d)" % fm for fm in GEN_FORMATS)
    todo.append((["-DBSFP_GEN_FORMATS=" + fmts], GEN_HEADER, "tuned"))
    for e in range(2, 9):
        for lo, hi in M_RANGES:
            ys = " ".join("Y(%d, %d)" % fm for fm in part_formats(e, lo, hi))
            zs = ys.replace("Y(", "Z(")
            for lst, macro, name, tag in ((ys, "-DBSFP_GEN_ADDMUL=", part_header(e, lo), "e%d_m%d" % (e, lo)),
                                          (zs, "-DBSFP_GEN_DIV=", div_header(e, lo), "div_e%d_m%d" % (e, lo))):
                path = os.path.join(GEN_DIR, name)
                if lst:
                    todo.append(([macro + lst], path, tag))
                elif not os.path.exists(path) or os.path.getmtime(path) < newest:
                    with open(path, "w") as fh:
                        fh.write("/* no formats of this part need printed netlists */\n")
    for e in range(2, 9):
        # both parts of an exponent width, for the units that span every fraction width
        for name, hdr in (("gen_e%d_all.cuh", part_header), ("gen_div_e%d_all.cuh", div_header)):
            path = os.path.join(GEN_DIR, name % e)
            if not os.path.exists(path) or os.path.getmtime(path) < newest:
                with open(path, "w") as fh:
                    fh.write("".join('#include "%s"\n' % hdr(e, lo) for lo, _ in M_RANGES))
    todo = [t for t in todo if not os.path.exists(t[1]) or os.path.getmtime(t[1]) < newest]
    with ThreadPoolExecutor(jobs or max(1, os.cpu_count() or 1)) as ex:
        for fut in [ex.submit(_generate_one, *t) for t in todo]:
            fut.result()
    return GEN_HEADER


def build(jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    generate(jobs)
    gen = glob.glob(os.path.join(GEN_DIR, "*.cuh"))
    newest = max(os.path.getmtime(p) for p in _deps() + gen)
    units = _units()
    todo = [(o, c) for o, c in units
            if not os.path.exists(os.path.join(BUILD, o)) or os.path.getmtime(os.path.join(BUILD, o)) < newest]
    jobs = jobs or max(1, os.cpu_count() or 1)

    def run(item):
        o, cmd = item
        out = os.path.join(BUILD, o)
        tmp = out + ".tmp"
        r = subprocess.run(cmd + ["-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            return o, r.stdout + r.stderr
        os.replace(tmp, out)
        return o, None

    # longest units first
    todo.sort(key=lambda t: (not t[0].startswith(("binop", "batch_opc")), t[0]))
    errors = []
    with ThreadPoolExecutor(jobs) as ex:
        for o, err in ex.map(run, todo):
            if err:
                errors.append("%s:\n%s" % (o, err))
            elif verbose:
                print("built", o, file=sys.stderr)
    if errors:
        raise RuntimeError("libbsfp build failed:\n" + "\n".join(errors))
    objs = [os.path.join(BUILD, o) for o, _ in units]
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(p) for p in objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                               "-Xlinker", "-rpath,/usr/local/cuda/lib64"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    print(LIB)
