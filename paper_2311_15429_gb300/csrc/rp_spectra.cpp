// Host FP64 construction of the kernel spectra of the FFT path.
//
// For the ordered pair (target t, source s) of equal spacing h and lag m, the
// space-time sampled Green's function of Eq. 11 is
//
//   G_m[k, k'] = h^3 T(m dt - R/c) / R,   T(u) = max(0, 1 - |u|/dt),
//
// with R = |o_t - o_s + h (i_t - i_s)| depending only on the index offset
// d = i_t - i_s in [-(n_s - 1), n_t - 1] per axis, so the sum over k' is a
// linear convolution.  Placing G at (d mod M) on a grid of M >= n_t + n_s - 1
// per axis makes the cyclic convolution of the zero-padded source equal the
// linear one on the target nodes (the Hockney construction).  For the self
// pair the R = 0 entry is the cell average C h^2 at lag 0 (zero at other
// lags).  The spectrum is computed in FP64 and stored in FP32, scaled by
// 1/(mx my mz) so that the inverse transform needs no further scaling.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "rp_internal.h"

namespace rp {

namespace {

using cd = std::complex<double>;

// Mixed-radix decimation-in-time FFT of length n (any n; radices 2, 3, 5 and
// a direct DFT for other prime factors), forward sign exp(-2 pi i jk/n).
class Fft1d {
  public:
    explicit Fft1d(int n) : n_(n), tw_(n), scratch_(n)
    {
        for (int j = 0; j < n; ++j) {
            const double a = -2.0 * M_PI * (double)j / (double)n;
            tw_[j] = cd(std::cos(a), std::sin(a));
        }
    }
    // in-place on data[0], data[stride], ..., data[(n-1)*stride]
    void run(cd *data, long long stride)
    {
        for (int j = 0; j < n_; ++j) scratch_[j] = data[j * stride];
        std::vector<cd> out(n_);
        rec(scratch_.data(), 1, n_, out.data());
        for (int j = 0; j < n_; ++j) data[j * stride] = out[j];
    }

  private:
    static int smallest_factor(int n)
    {
        for (int p = 2; p * p <= n; ++p)
            if (n % p == 0) return p;
        return n;
    }
    // out[k] = sum_j in[j*stride] W_n^{jk}; W_n^x = tw_[(x * (n_/n)) % n_]
    void rec(const cd *in, int stride, int n, cd *out)
    {
        if (n == 1) {
            out[0] = in[0];
            return;
        }
        const int p = smallest_factor(n), m = n / p;
        for (int r = 0; r < p; ++r) rec(in + r * stride, stride * p, m, out + r * m);
        std::vector<cd> tmp(n);
        const int step = n_ / n;
        for (int k = 0; k < m; ++k) {
            for (int q = 0; q < p; ++q) {
                const int kk = k + q * m;
                cd acc = 0.0;
                for (int r = 0; r < p; ++r) acc += out[r * m + k] * tw_[((long long)r * kk % n) * step];
                tmp[kk] = acc;
            }
        }
        for (int j = 0; j < n; ++j) out[j] = tmp[j];
    }

    int n_;
    std::vector<cd> tw_;
    std::vector<cd> scratch_;
};

}  // namespace

double cube_average_constant() { return 3.0 * std::log(2.0 + std::sqrt(3.0)) - 0.5 * M_PI; }

void build_kernel_spectrum(const double o_t[3], const int n_t[3], const double o_s[3], const int n_s[3],
                           double h, bool self_pair, int lag, double c, double dt, const int m[3],
                           bool real_out, float *out_real, float2 *out_cplx)
{
    const int mx = m[0], my = m[1], mz = m[2];
    const long long total = (long long)mx * my * mz;
    std::vector<cd> grid(total, cd(0.0, 0.0));   // [z][y][x]
    const double vol = h * h * h;
    const double cdt = c * dt;
    const double off[3] = {o_t[0] - o_s[0], o_t[1] - o_s[1], o_t[2] - o_s[2]};
    for (int dz = -(n_s[2] - 1); dz <= n_t[2] - 1; ++dz) {
        const double rz = off[2] + h * dz;
        const int iz = ((dz % mz) + mz) % mz;
        for (int dy = -(n_s[1] - 1); dy <= n_t[1] - 1; ++dy) {
            const double ry = off[1] + h * dy;
            const int iy = ((dy % my) + my) % my;
            for (int dx = -(n_s[0] - 1); dx <= n_t[0] - 1; ++dx) {
                const double rx = off[0] + h * dx;
                const int ix = ((dx % mx) + mx) % mx;
                const double R = std::sqrt(rx * rx + ry * ry + rz * rz);
                double val;
                if (self_pair && dx == 0 && dy == 0 && dz == 0) {
                    val = lag == 0 ? cube_average_constant() * h * h : 0.0;
                } else {
                    const double u = (double)lag - R / cdt;   // (m dt - R/c) / dt
                    const double T = std::fmax(0.0, 1.0 - std::fabs(u));
                    val = T > 0.0 ? vol * T / R : 0.0;
                }
                grid[((long long)iz * my + iy) * mx + ix] = cd(val, 0.0);
            }
        }
    }
    // 3D FFT: along x, then y, then z
    {
        Fft1d fx(mx);
        for (long long line = 0; line < (long long)my * mz; ++line) fx.run(grid.data() + line * mx, 1);
        Fft1d fy(my);
        for (int z = 0; z < mz; ++z)
            for (int x = 0; x < mx; ++x) fy.run(grid.data() + (long long)z * my * mx + x, mx);
        Fft1d fz(mz);
        for (long long xy = 0; xy < (long long)my * mx; ++xy) fz.run(grid.data() + xy, (long long)my * mx);
    }
    const int kx = mx / 2 + 1;
    const int ntile = (my + kTileY - 1) / kTileY;
    const long long cells = spec_cells(kx, my, mz);
    if (real_out) std::memset(out_real, 0, cells * sizeof(float));
    else std::memset(out_cplx, 0, cells * sizeof(float2));
    const double scale = 1.0 / (double)total;
    for (int k0 = 0; k0 < kx; ++k0)
        for (int kz = 0; kz < mz; ++kz)
            for (int ky = 0; ky < my; ++ky) {
                const cd v = grid[((long long)kz * my + ky) * mx + k0] * scale;
                const long long o = (((long long)k0 * ntile + ky / kTileY) * mz + kz) * kTileY + ky % kTileY;
                if (real_out)
                    out_real[o] = (float)v.real();
                else
                    out_cplx[o] = make_float2((float)v.real(), (float)v.imag());
            }
}

}  // namespace rp
