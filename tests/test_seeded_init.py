"""The device's seeded table initialisation computes what the generator
defines (CPU: the header's host side, compiled as plain C++, against
workload.kv_table_seeded; the device run is in test_gpu_kv.py)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2406_10158_gb300 import workload as wl

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2406_10158_gb300", "csrc")


@pytest.mark.parametrize("seed", [0, 0x5EED0001, (1 << 64) - 1])
def test_header_matches_the_generator(tmp_path, seed):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    nrec, nfields = 37, 5
    prog = tmp_path / "seeded.cpp"
    prog.write_text(f"""
#include <cstdio>
#include "seeded_init.cuh"
int main() {{
    const unsigned long long seed = {seed}ull;
    for (unsigned f = 0; f < {nfields}; ++f)
        for (unsigned k = 0; k < {nrec}; ++k)
            std::printf("%llu %llu\\n",
                        (unsigned long long)gcc::seeded::slot_lo(seed, k, f, {nfields}),
                        (unsigned long long)gcc::seeded::slot_hi(seed, k, f, {nfields}));
    return 0;
}}
""")
    exe = tmp_path / "seeded"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(prog)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = np.array([int(v) for v in out], dtype=np.uint64).reshape(nfields, nrec, 2)
    assert np.array_equal(got[..., 0], wl.kv_table_seeded(seed, nrec, nfields, 8))
    assert np.array_equal(got, wl.kv_table_seeded(seed, nrec, nfields, 16))


def test_sixteen_byte_values_use_ten_bytes():
    t = wl.kv_table_seeded(9, 1000, 3, 16)
    assert t.shape == (3, 1000, 2)
    assert (t[..., 1] >> np.uint64(16) == 0).all()
    assert len(np.unique(t[..., 1])) > 900         # bytes 8-9 vary
    assert np.array_equal(t[..., 0], wl.kv_table_splitmix(9, 1000, 3))
