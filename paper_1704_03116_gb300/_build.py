"""Build of the CUDA library libdope.so (sm_103a), in-tree.

Four translation units, compiled in parallel by nvcc for sm_103a only and
linked into one shared library: csrc/dope.cu (kernels in csrc/*.cuh, the
solver C-ABI), csrc/dope_big.cu (the larger-kernel instantiations),
csrc/dope_server.cu (the request server, host code) and
csrc/dope_potentials.cu (the whole-image potentials).  It links the CUDA runtime statically and has no PyTorch
dependency (the C-ABI takes plain pointers).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", "dope.cu"), os.path.join(HERE, "csrc", "dope_big.cu"),
       os.path.join(HERE, "csrc", "dope_server.cu"), os.path.join(HERE, "csrc", "dope_potentials.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("dope_kernels.cuh", "dope_internal.h", "dope_overlap.cuh",
                                                       "dope_nsm.cuh", "dope_big.h")] + \
    [os.path.join(ROOT, "include", h) for h in ("dope.h", "dope_potentials.h")]
OBJDIR = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libdope.so")
LIB_CHECKED = os.path.join(HERE, "libdope_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force=False, verbose=False, checked=False):
    """Compile libdope.so if it is missing or older than its sources.  With
    checked=True, libdope_checked.so instead: the same library with
    DOPE_CHECKED, every shared-memory index of the block solver and the
    resident kernel tested against its array (dope_check_status)."""
    lib = LIB_CHECKED if checked else LIB
    objdir = os.path.join(OBJDIR, "checked") if checked else OBJDIR
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in DEPS)):
        return lib
    os.makedirs(objdir, exist_ok=True)
    common = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I" + os.path.join(ROOT, "include")]
    if checked:
        common.append("-DDOPE_CHECKED")
    if verbose:
        common.insert(1, "-Xptxas=-v")
    objs, procs = [], []
    for src in SRC:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        objs.append(obj)
        procs.append(subprocess.Popen([*common, "-c", "-o", obj, src], stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    failed = False
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            sys.stderr.write(out + err)
            failed = True
        elif verbose:
            sys.stderr.write(err)
    if failed:
        raise RuntimeError("nvcc failed building libdope.so")
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking " + os.path.basename(lib))
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
