"""Build liblbo.so (the C ABI of include/lbo.h) from csrc/*.cu with nvcc for
sm_103a.  Translation units compile in parallel into _build/ (a source may
ask to be compiled once per set of -D flags, see _units), then link into
paper_2503_09580_gb300/_lib/liblbo.so."""
import concurrent.futures
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "liblbo.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _units():
    """(source, object name, extra flags) per translation unit.  A source whose
    first line reads `// build-variants: A=1:B=2 A=1:B=3 ...` is compiled once
    per entry, each entry's NAME=VALUE pairs passed as -D flags."""
    units = []
    for src in _sources():
        base = os.path.basename(src)[:-3]
        with open(src) as fh:
            first = fh.readline()
        tag = "// build-variants:"
        if first.startswith(tag):
            for entry in first[len(tag):].split():
                defs = entry.split(":")
                name = base + "_" + "_".join(d.split("=", 1)[1] for d in defs)
                units.append((src, name, ["-D" + d for d in defs]))
        else:
            units.append((src, base, []))
    return units


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "lbo.h"))
    return hs


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def _compile(unit, force):
    src, name, extra = unit
    obj = os.path.join(BUILD, name + ".o")
    if (not force and os.path.exists(obj)
            and os.path.getmtime(obj) >= max(os.path.getmtime(src), _newest(_headers()))):
        return obj
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj


def build(force=False, verbose=False):
    """Compile every CUDA translation unit and link liblbo.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    units = _units()
    # the slowest units first, so that the parallel build ends with short ones
    units.sort(key=lambda u: (not u[2], u[1]))
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda u: _compile(u, force), units))
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
