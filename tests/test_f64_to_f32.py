"""The integer-ALU conversions of the device code (csrc/f64cvt.h) against the
host's own conversions, bit for bit. Binary64 -> binary32 (round to nearest,
ties to even): random bit patterns over every exponent, and the boundaries
where a mistake would show: ties with even and odd last bits, a carry out of
the fraction, the largest finite value and overflow, the smallest normal
value and the subnormal range, signed zeros, infinities and NaNs. Binary32 ->
binary64 (exact): a stride through all 2^32 patterns and every exponent's
boundary fractions."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER_DIR = os.path.join(os.path.dirname(HERE), "paper_1009_3308_gb300", "csrc")

PROGRAM = r"""
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <initializer_list>
#include "f64cvt.h"

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t next() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }
static long bad = 0, n = 0;
static void check(uint64_t bits) {
    double x; std::memcpy(&x, &bits, 8);
    const float a = sph::f64_to_f32_rn(x), b = static_cast<float>(x);
    uint32_t ua, ub; std::memcpy(&ua, &a, 4); std::memcpy(&ub, &b, 4);
    ++n;
    if (std::isnan(b) ? !std::isnan(a) : ua != ub) {
        if (bad < 10) std::printf("mismatch %016llx: %08x vs %08x\n", (unsigned long long)bits, ua, ub);
        ++bad;
    }
}
int main() {
    for (int i = 0; i < 2000000; ++i) check(next());
    // random fractions at every binary64 exponent
    for (uint64_t e = 0; e < 2048; ++e)
        for (int i = 0; i < 200; ++i) check((next() & 0x800FFFFFFFFFFFFFull) | (e << 52));
    // ties and their neighbours at the binary32 rounding position, every
    // exponent around the binary32 range
    for (uint64_t e = 1023 - 160; e <= 1023 + 130; ++e)
        for (int i = 0; i < 64; ++i) {
            const uint64_t frac = next() & 0x000FFFFFE0000000ull;   // 23 kept bits
            for (int64_t d : {-1, 0, 1})
                for (uint64_t sg : {0ull, 1ull << 63})
                    check(sg | (e << 52) | ((frac | 0x10000000ull) + uint64_t(d)));
            check((e << 52) | 0x000FFFFFE0000000ull | 0x10000000ull);   // all ones + tie: carry
            check((e << 52) | 0x000FFFFFF0000000ull);                   // above the tie with all ones
        }
    const double special[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 3.4028234663852886e38, 3.4028235677973366e38,
                              3.4028235677973362e38, 1e39, -1e39, 1.1754943508222875e-38, 1.1754942807573643e-38,
                              1.401298464324817e-45, 7.006492321624085e-46, 7.006492321624087e-46, 1e-50, 4.9e-324};
    for (double x : special) { uint64_t b; std::memcpy(&b, &x, 8); check(b); check(b ^ (1ull << 63)); }
    // binary32 -> binary64 (exact): every 61st bit pattern, and every
    // exponent with its boundary fractions
    long bad2 = 0, n2 = 0;
    auto check2 = [&](uint32_t u) {
        float x; std::memcpy(&x, &u, 4);
        const double a = sph::f32_to_f64(x), b = static_cast<double>(x);
        uint64_t ua, ub; std::memcpy(&ua, &a, 8); std::memcpy(&ub, &b, 8);
        ++n2;
        if (std::isnan(b) ? !std::isnan(a) : ua != ub) {
            if (bad2 < 10) std::printf("widen mismatch %08x: %016llx vs %016llx\n", u, (unsigned long long)ua, (unsigned long long)ub);
            ++bad2;
        }
    };
    for (uint64_t u = 0; u <= 0xFFFFFFFFull; u += 61) check2(uint32_t(u));
    for (uint32_t e = 0; e < 256; ++e)
        for (uint32_t fr : {0u, 1u, 0x400000u, 0x7FFFFFu})
            for (uint32_t sg : {0u, 0x80000000u}) check2(sg | (e << 23) | fr);
    std::printf("checked %ld mismatches %ld; widened %ld mismatches %ld\n", n, bad, n2, bad2);
    return bad != 0 || bad2 != 0;
}
"""


def test_integer_conversion_matches_ieee_round_to_nearest(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    src = tmp_path / "cvt.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "cvt"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert "mismatches 0;" in r.stdout and r.stdout.strip().endswith("mismatches 0")
