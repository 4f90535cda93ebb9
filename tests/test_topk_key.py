"""The top-K passes form the radix key of an FP32 residual from the float's
bits with integer operations (csrc/topk_key.cuh).  It must equal the bit
pattern of the FP64 value (double)|v|, the key the FP64 passes and the oracle
rank by, for every float that is not a NaN.  The header's function is compiled
for the host and compared with the C conversion on all 2^31 magnitudes (zero,
subnormals, normal numbers, infinity)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2510_02156_gb300", "csrc", "topk_key.cuh")

SRC = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include <stdio.h>
#include <string.h>
#include "%s"
int main(void) {
    unsigned long long bad = 0, checked = 0;
    for (unsigned long long w = 0; w <= 0x7f800000ull; ++w) {
        const unsigned u = (unsigned)w;
        float f;
        memcpy(&f, &u, 4);
        const double d = (double)f;
        unsigned long long k;
        memcpy(&k, &d, 8);
        k &= 0x7fffffffffffffffull;
        /* the sign bit is dropped: negative floats map to the same key */
        if (topk_key_f32_bits(u) != k || topk_key_f32_bits(u | 0x80000000u) != k) {
            if (bad < 5) printf("mismatch %%08x\n", u);
            ++bad;
        }
        ++checked;
    }
    printf("%%llu %%llu\n", checked, bad);
    return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_integer_key_equals_the_fp64_key_of_every_float(tmp_path):
    src = tmp_path / "key.c"
    src.write_text(SRC % os.path.abspath(HEADER))
    exe = tmp_path / "key"
    subprocess.run(["gcc", "-O2", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    checked, bad = map(int, out.stdout.split()[-2:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert checked == 0x7f800000 + 1
