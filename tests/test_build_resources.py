"""Resource properties of the hot kernels, from ptxas's report of an sm_103a build (no GPU).

The 4^4-block SAP sweep fits two 256-thread CTAs per SM only with at most 128
registers per thread, and it is only fast without local memory (the generic
staged kernel kept its direction tables there); the cluster-split Arnoldi step
runs 512-thread CTAs.  A change that breaks one of these shows up here before it
reaches a GPU."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1307_6101_gb300", "csrc")


def _ptxas_report(src):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
               "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v", "-c",
               os.path.join(CSRC, src), "-o", os.path.join(d, "k.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = {}
    name = None
    for ln in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", ln)
        if m:
            name = m.group(1)
            out[name] = {}
            continue
        if name is None:
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", ln)
        if m:
            out[name].update(stack=int(m.group(1)), spill_st=int(m.group(2)), spill_ld=int(m.group(3)))
        m = re.search(r"Used (\d+) registers", ln)
        if m:
            out[name]["regs"] = int(m.group(1))
    return out


def test_fine_sap_4x4_kernel_resources():
    rep = _ptxas_report("fine.cu")
    b4 = {k: v for k, v in rep.items() if "k_fine_sap_b4" in k and "k_fine_sap_b4_eo" not in k}
    assert len(b4) == 2                                  # FP16 and FP32 storage
    for k, v in b4.items():
        assert v["regs"] <= 128, (k, v)
        assert v["stack"] == 0 and v["spill_st"] == 0 and v["spill_ld"] == 0, (k, v)
    # the Schur variant: two 128-thread CTAs per SM, no local memory
    eo = {k: v for k, v in rep.items() if "k_fine_sap_b4_eo" in k}
    assert len(eo) == 2
    for k, v in eo.items():
        assert v["regs"] * 128 * 2 <= 65536, (k, v)
        assert v["stack"] == 0 and v["spill_st"] == 0 and v["spill_ld"] == 0, (k, v)


def test_tensor_core_kernels_resources():
    """The tensor-core coarse stencil and restriction keep their fragments and accumulators in
    registers (no local memory).  The restriction's largest CTA (N <= 32 test vectors, 4 tiles x 4
    k-splits = 512 threads) fits an SM's registers; the coarse stencil's launcher rejects CTAs above
    the kernel's register-limited maximum, and the largest CTA of the 56-dof levels (7 tiles x 4
    k-splits = 896 threads) must fit (registers are allocated per warp in units of 8 per thread)."""
    for src, name, threads in (("coarse_tc.cu", "k_coarse_apply_tc", 896), ("transfer_tc.cu", "k_restrict_tc", 512)):
        rep = _ptxas_report(src)
        ks = {k: v for k, v in rep.items() if name in k}
        assert ks, (src, list(rep))
        for k, v in ks.items():
            assert v["spill_st"] == 0 and v["spill_ld"] == 0, (k, v)
            assert ((v["regs"] + 7) // 8 * 8) * threads <= 65536, (k, v)


def test_arnoldi_cluster_kernel_resources():
    rep = _ptxas_report("krylov.cu")
    cl = {k: v for k, v in rep.items() if "k_arnoldi_cl" in k}
    assert len(cl) == 2                                  # FP32 and FP64 vectors
    for k, v in cl.items():
        assert v["regs"] * 512 <= 65536, (k, v)          # one 512-thread CTA fits an SM's registers


def test_coarse_sap_eight_rows_per_thread_fits_3024_row_blocks():
    """The 48^3x96 hierarchy's widened level-2 SAP blocks have 2*3*3*3 sites x 56 dof = 3024 rows: at
    eight rows per thread, 378 threads (12 warps) of every variant must fit an SM's 65536 registers
    (registers are allocated per warp in units of 8 per thread)."""
    rep = _ptxas_report("coarse.cu")
    r8 = {k: v for k, v in rep.items() if "k_coarse_sap" in k and "Li8E" in k}
    assert len(r8) == 3                                  # FP64, FP32, FP32 on FP16 blocks
    warps = (3024 // 8 + 31) // 32
    for k, v in r8.items():
        assert ((v["regs"] + 7) // 8 * 8) * 32 * warps <= 65536, (k, v)
