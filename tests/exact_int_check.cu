// Host check of the integer-pipe exact helpers of nb_exact.cuh against the host's
// IEEE arithmetic (correctly rounded by IEEE 754): div3_int, div15_int and
// mul3_int must return the bits of y / 6, y / 24, y / 120 and 3 y 2^s wherever they
// accept y, and ds_split_int the bits of (float)x and (float)(x - hi). Random and
// edge significands over the whole accepted exponent windows.
// Usage: exact_int_check [cases]; exits non-zero on a mismatch.
//        exact_int_check quantise < records: for each record of five doubles
//        (candidate, dt_old, t_new, dt_max, dt_min) on standard input (after an
//        int64 count) writes the bit-pattern quantiser's step as a double.
//        exact_int_check aarseth < records: for each record (A, K, P, Q, eta) of
//        FP64 squared norms writes (decided, bits of the power of two) as the
//        corrector derives them: FP32 copies, their square roots, the FP32
//        estimate and its window.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "nb_exact.cuh"
#include "nb_hermite.cuh"

using namespace nb;

static unsigned long long sm_state = 0x2007110812345678ull;
static unsigned long long splitmix()
{
    unsigned long long z = (sm_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int fails = 0;
static void check(const char *what, double y, bool ok, double got, double ref)
{
    if (!ok) return;
    if (dbits(got) != dbits(ref)) {
        if (fails < 10)
            std::printf("MISMATCH %s y=%a got=%a ref=%a\n", what, y, got, ref);
        ++fails;
    }
}

static int quantise_mode()
{
    long long n = 0;
    if (std::fread(&n, 8, 1, stdin) != 1 || n < 0) return 2;
    for (long long q = 0; q < n; ++q) {
        double r[5];
        if (std::fread(r, 8, 5, stdin) != 5) return 2;
        const double dt = quantise_bits(pow2_floor_bits(r[0]), dpositive(r[0]), r[1], r[2], r[3], r[4]);
        if (std::fwrite(&dt, 8, 1, stdout) != 1) return 2;
    }
    return 0;
}

static int aarseth_mode()
{
    long long n = 0;
    if (std::fread(&n, 8, 1, stdin) != 1 || n < 0) return 2;
    for (long long q = 0; q < n; ++q) {
        double r[5];
        if (std::fread(r, 8, 5, stdin) != 5) return 2;
        long long qb = 0;
        bool decided = norm2_in_range(r[0]) && norm2_in_range(r[1]) && norm2_in_range(r[2]) && norm2_in_range(r[3]);
        if (decided) {
            const float fA = (float)r[0], fK = (float)r[1], fP = (float)r[2], fQ = (float)r[3];
            decided = aarseth_estimate(std::sqrt(fA), std::sqrt(fK), std::sqrt(fP), std::sqrt(fQ), fK, fP,
                                       (float)r[4], qb);
        }
        const double out[2] = {decided ? 1.0 : 0.0, dfrom(qb)};
        if (std::fwrite(out, 8, 2, stdout) != 2) return 2;
    }
    return 0;
}

// The corrector's FP32 norms: records of the four vectors' FP64 components (a, k,
// a2p, a3; 12 values) and eta; RN32 copies on the integer pipe, squares flushed
// below 2^-126, (x^2 + y^2) + z^2, then the estimate. Writes (decided, power of two).
static int aarseth32_mode()
{
    long long n = 0;
    if (std::fread(&n, 8, 1, stdin) != 1 || n < 0) return 2;
    for (long long q = 0; q < n; ++q) {
        double r[13];
        if (std::fread(r, 8, 13, stdin) != 13) return 2;
        float S[4];
        bool ok = true;
        for (int v = 0; v < 4; ++v) {
            float c[3];
            for (int k = 0; k < 3; ++k) ok = rn32_int(r[3 * v + k], c[k]) && ok;
            S[v] = (sq_ftz(c[0]) + sq_ftz(c[1])) + sq_ftz(c[2]);
            ok = ok && norm2_f32_in_range(S[v]);
        }
        long long qb = 0;
        bool decided = ok && aarseth_estimate(std::sqrt(S[0]), std::sqrt(S[1]), std::sqrt(S[2]), std::sqrt(S[3]),
                                              S[1], S[2], (float)r[12], qb);
        const double out[2] = {decided ? 1.0 : 0.0, dfrom(qb)};
        if (std::fwrite(out, 8, 2, stdout) != 2) return 2;
    }
    return 0;
}

// rn32_int against the host's double-to-float conversion (subnormal floats
// flushed) on random doubles of every exponent below 2^60.
static long long rn32_check(long long cases)
{
    long long bad = 0;
    for (long long n = 0; n < cases; ++n) {
        const unsigned long long r = splitmix();
        const int E = (int)(splitmix() % (1023 + 60));
        const double y = dfrom((long long)((r & (1ull << 63)) | ((unsigned long long)E << 52) | (r & ((1ull << 52) - 1))));
        float f = 1.f;
        const bool ok = rn32_int(y, f);
        float ref = (float)y;
        if (std::fabs(ref) < 1.17549435e-38f) ref = 0.f;
        if (!ok || (f != ref) || (f == 0.f && ref != 0.f)) {
            if (bad < 5) std::printf("MISMATCH rn32 y=%a got=%a ref=%a\n", y, (double)f, (double)ref);
            ++bad;
        }
    }
    for (double big : {0x1p60, -0x1p61, 1.0 / 0.0}) {
        float f;
        if (rn32_int(big, f)) ++bad;
    }
    return bad;
}

int main(int argc, char **argv)
{
    if (argc > 1 && std::string(argv[1]) == "quantise") return quantise_mode();
    if (argc > 1 && std::string(argv[1]) == "aarseth") return aarseth_mode();
    if (argc > 1 && std::string(argv[1]) == "aarseth32") return aarseth32_mode();
    const long long cases = argc > 1 ? std::atoll(argv[1]) : 4000000;
    const unsigned long long edges[] = {0ull, 1ull, 2ull, (1ull << 52) - 1, (1ull << 52) - 2, (1ull << 51),
                                        (1ull << 51) - 1, (1ull << 51) + 1, (1ull << 50), (1ull << 49),
                                        (3ull << 49) - 1, (3ull << 49), (7ull << 49) - 1, (7ull << 49),
                                        (5ull << 48), 0x5555555555555ull, 0xAAAAAAAAAAAAAull,
                                        0x1111111111111ull, 0x8888888888888ull, 0x2AAAAAAAAAAAAull};
    long long accepted = 0, declined = 0;
    for (long long n = 0; n < cases; ++n) {
        const unsigned long long r = splitmix();
        unsigned long long mant = r & ((1ull << 52) - 1);
        if ((n & 7) == 0) mant = edges[(r >> 52) % (sizeof edges / sizeof edges[0])] ^ ((r >> 60) & 1);
        const int E = (int)(splitmix() % 2047);   // every biased exponent but inf/NaN
        const unsigned long long sign = (splitmix() & 1) << 63;
        const double y = dfrom((long long)(sign | ((unsigned long long)E << 52) | mant));
        double out;
        bool ok;
        ok = div3_int(y, 1, out);
        check("y/6", y, ok, out, y / 6.0);
        accepted += ok; declined += !ok;
        ok = div3_int(y, 3, out);
        check("y/24", y, ok, out, y / 24.0);
        ok = div3_int(y, 0, out);
        check("y/3", y, ok, out, y / 3.0);
        ok = div15_int(y, 3, out);
        check("y/120", y, ok, out, y / 120.0);
        ok = div15_int(y, 0, out);
        check("y/15", y, ok, out, y / 15.0);
        for (int s = 0; s <= 3; ++s) {
            ok = mul3_int(y, s, out);
            check("3y*2^s", y, ok, out, (3.0 * y) * std::ldexp(1.0, s));
        }
        unsigned hi, lo;
        if (ds_split_int(y, hi, lo)) {
            const float h = (float)y;
            const float l = (float)(y - (double)h);
            unsigned hb, lb;
            std::memcpy(&hb, &h, 4);
            std::memcpy(&lb, &l, 4);
            if (hi != hb || lo != lb) {
                if (fails < 10) std::printf("MISMATCH ds_split y=%a hi %08x/%08x lo %08x/%08x\n", y, hi, hb, lo, lb);
                ++fails;
            }
        }
    }
    fails += (int)rn32_check(cases / 4);
    std::printf("cases %lld (div3 accepted %lld, declined %lld), mismatches %d\n", cases, accepted, declined, fails);
    return fails ? 1 : 0;
}
