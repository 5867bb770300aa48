"""Build helper for the plain-C client of libfr.so (tests/c_client/render_request.c)."""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c_client", "render_request.c")
ROOT = os.path.dirname(HERE)


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.isdir(os.path.join(cand, "include")):
            return cand
    nvcc = shutil.which("nvcc")
    return os.path.dirname(os.path.dirname(nvcc)) if nvcc else "/usr/local/cuda"


def build(out_dir: str) -> str:
    """Compile and link the client against the in-tree libfr.so with gcc (C99)."""
    from paper_2102_01747_gb300 import build as B

    lib = B.build()
    cuda = cuda_home()
    exe = os.path.join(out_dir, "render_request")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O2",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           SRC, "-o", exe, "-L", libdir, "-lfr", "-Wl,-rpath," + libdir,
           "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe
