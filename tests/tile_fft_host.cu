// Host harness for the two-stage tile transform of rp_fft.cuh: the stage
// functions are host-callable, so their index logic and arithmetic are run
// here task by task (the tasks of a stage touch disjoint rows, so running
// them one after another gives what the warp computes) on seeded inputs and
// compared with the plain DFT sum in double precision.  Prints one line per
// case: "name rel_l2".
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "../paper_2311_15429_gb300/csrc/rp_fft.cuh"

using namespace rp;

template <int B, bool INV, bool HALF, int SP, int SC>
static double run_case(int nin, unsigned seed)
{
    const int M = 16 * B;
    std::vector<float2> tw(M), T((size_t)M * SP + (size_t)16 * SC * M + 64);
    for (int j = 0; j < M; ++j)
        tw[j] = make_float2((float)std::cos(-2.0 * M_PI * j / M), (float)std::sin(-2.0 * M_PI * j / M));
    std::mt19937 g(seed);
    std::normal_distribution<float> nd;
    std::vector<double> xr((size_t)M * 16), xi((size_t)M * 16);
    for (int p = 0; p < M; ++p)
        for (int c = 0; c < 16; ++c) {
            const float a = nd(g), b = nd(g);
            const bool zero = p >= nin || (HALF && p >= M / 2);
            // rows the transform must not read hold garbage
            T[(size_t)p * SP + (size_t)c * SC] = zero ? make_float2(1e30f, -1e30f) : make_float2(a, b);
            xr[(size_t)p * 16 + c] = zero ? 0.0 : a;
            xi[(size_t)p * 16 + c] = zero ? 0.0 : b;
        }
    for (int n2 = 0; n2 < B; ++n2)
        for (int c = 0; c < 16; ++c) tile_stage1<B, INV, HALF, SP, SC>(T.data(), tw.data(), nin, c, n2);
    for (int k1 = 0; k1 < 16; ++k1)
        for (int c = 0; c < 16; ++c) tile_stage2<B, INV, SP, SC>(T.data(), c, k1);
    const double sg = INV ? 1.0 : -1.0;
    double num = 0.0, den = 0.0;
    for (int c = 0; c < 16; ++c)
        for (int k = 0; k < M; ++k) {
            double re = 0.0, im = 0.0;
            for (int n = 0; n < M; ++n) {
                const double ang = sg * 2.0 * M_PI * (double)((long long)n * k % M) / M;
                re += xr[(size_t)n * 16 + c] * std::cos(ang) - xi[(size_t)n * 16 + c] * std::sin(ang);
                im += xr[(size_t)n * 16 + c] * std::sin(ang) + xi[(size_t)n * 16 + c] * std::cos(ang);
            }
            const float2 got = T[(size_t)tile_row<B>(k) * SP + (size_t)c * SC];
            num += (got.x - re) * (got.x - re) + (got.y - im) * (got.y - im);
            den += re * re + im * im;
        }
    return std::sqrt(num / den);
}

int main()
{
    std::printf("fwd64 %.6e\n", run_case<4, false, false, 16, 1>(64, 1));
    std::printf("inv64 %.6e\n", run_case<4, true, false, 16, 1>(64, 2));
    std::printf("half64_nin29 %.6e\n", run_case<4, false, true, 16, 1>(29, 3));
    std::printf("fwd96 %.6e\n", run_case<6, false, false, 16, 1>(96, 4));
    std::printf("inv96 %.6e\n", run_case<6, true, false, 16, 1>(96, 5));
    std::printf("half96_nin48 %.6e\n", run_case<6, false, true, 16, 1>(48, 6));
    std::printf("fwd96_nin50 %.6e\n", run_case<6, false, false, 16, 1>(50, 7));
    std::printf("fwd128 %.6e\n", run_case<8, false, false, 16, 1>(128, 8));
    std::printf("inv128 %.6e\n", run_case<8, true, false, 16, 1>(128, 9));
    std::printf("fwd192 %.6e\n", run_case<12, false, false, 16, 1>(192, 10));
    std::printf("half192_nin77 %.6e\n", run_case<12, false, true, 16, 1>(77, 11));
    std::printf("rows96_sc97_half %.6e\n", run_case<6, false, true, 1, 97>(41, 12));
    std::printf("rows96_sc97_inv %.6e\n", run_case<6, true, false, 1, 97>(96, 13));
    std::printf("cols96_sp17_inv %.6e\n", run_case<6, true, false, 17, 1>(96, 14));
    std::printf("cols96_sp49_half %.6e\n", run_case<6, false, true, 49, 1>(48, 15));
    std::printf("rows128_sc129_inv %.6e\n", run_case<8, true, false, 1, 129>(128, 16));
    std::printf("inv32 %.6e\n", run_case<2, true, false, 16, 1>(32, 17));
    std::printf("inv48 %.6e\n", run_case<3, true, false, 16, 1>(48, 18));
    std::printf("fwd48_nin24 %.6e\n", run_case<3, false, false, 16, 1>(24, 19));
    std::printf("rows192_sc193_inv %.6e\n", run_case<12, true, false, 1, 193>(192, 20));
    std::printf("cols192_sp17_inv %.6e\n", run_case<12, true, false, 17, 1>(192, 21));
    return 0;
}
