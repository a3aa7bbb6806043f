"""Host logic of the batched plan (work list, table and coefficient pools)
run on the CPU under AddressSanitizer and UBSan, with the CUDA runtime calls
replaced by host-memory stand-ins (tests/hoststub/)."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "paper_1612_09001_gb300", "csrc", "batched_api.cu")


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_batched_plan_host_code_under_asan():
    src = open(SRC).read()
    src = src.replace('#include <cuda_runtime.h>', '#include "stub_cuda.h"')
    src = src.replace('#include "dpd_batched.cuh"', '#include "stub_batched.h"')
    src = src.replace('#include "../../include/dpd.h"', '#include "dpd.h"')
    src = re.sub(r"^namespace dpd \{\n.*?^\}  // namespace dpd\n", "", src, count=1, flags=re.S | re.M)
    tmp = tempfile.mkdtemp(prefix="asan_")
    try:
        api = os.path.join(tmp, "api_host.cpp")
        with open(api, "w") as f:
            f.write(src)
        exe = os.path.join(tmp, "t")
        cmd = ["g++", "-std=c++17", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
               "-I", os.path.join(HERE, "hoststub"), "-I", os.path.join(ROOT, "include"),
               "-I", os.path.join(ROOT, "paper_1612_09001_gb300", "csrc"),
               api, os.path.join(HERE, "hoststub", "plan_main.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 and re.search(r"-lasan|-lubsan|libasan|libubsan", r.stderr or ""):
            pytest.skip("AddressSanitizer runtime not available")
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "count 8 rc 0" in r.stdout and "ERROR" not in r.stderr, r.stdout + r.stderr
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
