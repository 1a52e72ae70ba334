"""The bounds-checked variant of the library (-DRSX_CHECKED) compiles: the translation units
whose FFT-pass kernels carry the index checks, cross-compiled for sm_103a (no GPU needed)."""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2405_01522_gb300 import build as b


@pytest.mark.skipif(shutil.which(b.NVCC) is None and not os.path.exists(b.NVCC), reason="nvcc not available")
def test_checked_translation_units_compile(tmp_path):
    srcs = ["poisson_p1.cu", "poisson_p3.cu", "api.cu"]

    def one(src):
        cmd = [b.NVCC] + b.ARCH + b.FLAGS + ["-DRSX_CHECKED", "-c", os.path.join(b.CSRC, src),
                                              "-o", str(tmp_path / (src + ".o"))]
        return subprocess.run(cmd, capture_output=True, text=True)

    with ThreadPoolExecutor(len(srcs)) as ex:
        res = list(ex.map(one, srcs))
    for src, r in zip(srcs, res):
        assert r.returncode == 0, f"{src}: {r.stderr[-2000:]}"
