"""The two-stage tile transform of the FFT passes (rp_fft.cuh), run on the
host: its stage functions compiled by nvcc for the CPU (tile_fft_host.cu)
and compared, for every padded length it serves (M = 64, 96, 128, 192),
forward and inverse, the zero-padded input (HALF) and the strided layouts
of the plane passes (the 192-point inverse plane pass's row and column tiles
included), and the odd and short lengths of the MAC's inverse column
transform (M = 32, 48), with the plain DFT sum in double precision.  The bar,
1e-6 rel-L2, is the FP32 transform's (measured 7e-8 to 1e-7)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tile_transform_matches_the_dft(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                    else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "tile_fft_host")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", os.path.join(HERE, "tile_fft_host.cu"), "-o", exe],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    errs = dict((ln.split()[0], float(ln.split()[1])) for ln in out.strip().splitlines())
    assert len(errs) == 21, out
    for name, e in errs.items():
        assert e <= 1e-6, (name, e)
