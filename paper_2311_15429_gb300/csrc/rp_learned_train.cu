// Learned far field, host side: synthetic training histories, the data set
// of (network row, target) pairs, the Adam training loop and the validation
// error of a trained network on a given pair geometry.
//
// A history is kLGauss Gaussians on the source grid with amplitudes
// A_g(t) = a (1 + e sin(w t + phi)) and the continuity-consistent current
// J = sum_g dA_g/dt / (4 pi) grad Phi_g (Phi_g the potential of Gaussian g),
// seen from a target box at distance Rc in direction n.  Its targets are the
// direct retarded sums (Eqs. 2, 7, 8) at the canonical nodes; its rows are
// the canonical moment windows (rp_learned_data.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rp_learned.h"
#include "rp_learned_data.h"
#include "rp_learned_train.h"

namespace rp {

namespace {

struct Rng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    double uniform(double a, double b) { return a + (b - a) * uniform(); }
    double normal()
    {
        const double u1 = std::max(uniform(), 1e-300), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    }
};

template <class T>
struct DevBuf {
    T *p = nullptr;
    cudaError_t alloc(size_t n)
    {
        free();
        return cudaMalloc(reinterpret_cast<void **>(&p), std::max<size_t>(n, 1) * sizeof(T));
    }
    void free()
    {
        if (p) cudaFree(p);
        p = nullptr;
    }
    ~DevBuf() { free(); }
};

}  // namespace

void canonical_frame(const double n_in[3], double R[9])
{
    double n[3] = {n_in[0], n_in[1], n_in[2]};
    const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (double &v : n) v /= nn;
    int k = 0;   // the axis least aligned with n (lowest index on ties)
    for (int i = 1; i < 3; ++i)
        if (std::fabs(n[i]) < std::fabs(n[k])) k = i;
    double e[3] = {0.0, 0.0, 0.0};
    e[k] = 1.0;
    const double en = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];
    double u[3] = {e[0] - en * n[0], e[1] - en * n[1], e[2] - en * n[2]};
    const double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (double &v : u) v /= un;
    const double w[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};
    for (int i = 0; i < 3; ++i) {
        R[i] = n[i];
        R[3 + i] = u[i];
        R[6 + i] = w[i];
    }
}

void canonical_nodes(const double Lt[3], double nodes[kLOut][3])
{
    const double hw = 0.5 * std::sqrt(Lt[0] * Lt[0] + Lt[1] * Lt[1] + Lt[2] * Lt[2]);
    double g[kLNodes];
    for (int a = 0; a < kLNodes; ++a) g[a] = -hw * std::cos((2.0 * a + 1.0) * M_PI / (2.0 * kLNodes));
    int i = 0;
    for (int c = 0; c < kLNodes; ++c)
        for (int b = 0; b < kLNodes; ++b)
            for (int a = 0; a < kLNodes; ++a, ++i) {
                nodes[i][0] = g[a];
                nodes[i][1] = g[b];
                nodes[i][2] = g[c];
            }
}

double canonical_half_width(const double Lt[3])
{
    return 0.5 * std::sqrt(Lt[0] * Lt[0] + Lt[1] * Lt[1] + Lt[2] * Lt[2]);
}

static void lagrange(const double *g, int p, double x, double *w)
{
    for (int a = 0; a < p; ++a) {
        double v = 1.0;
        for (int b = 0; b < p; ++b)
            if (b != a) v *= (x - g[b]) / (g[a] - g[b]);
        w[a] = v;
    }
}

void reinterp_matrix(const double Lt[3], const double R[9], const double ct[3], const std::vector<double> *tnodes,
                     std::vector<float> &P)
{
    const double hw = canonical_half_width(Lt);
    double g[kLNodes];
    for (int a = 0; a < kLNodes; ++a) g[a] = -hw * std::cos((2.0 * a + 1.0) * M_PI / (2.0 * kLNodes));
    const int px = (int)tnodes[0].size(), py = (int)tnodes[1].size(), pz = (int)tnodes[2].size();
    P.assign((size_t)px * py * pz * kLOut, 0.0f);
    int b = 0;
    for (int k = 0; k < pz; ++k)
        for (int j = 0; j < py; ++j)
            for (int i = 0; i < px; ++i, ++b) {
                const double d[3] = {tnodes[0][i] - ct[0], tnodes[1][j] - ct[1], tnodes[2][k] - ct[2]};
                double xc[3];
                for (int r = 0; r < 3; ++r) xc[r] = R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2];
                double wa[kLNodes], wb[kLNodes], wc[kLNodes];
                lagrange(g, kLNodes, xc[0], wa);
                lagrange(g, kLNodes, xc[1], wb);
                lagrange(g, kLNodes, xc[2], wc);
                int a = 0;
                for (int c3 = 0; c3 < kLNodes; ++c3)
                    for (int b3 = 0; b3 < kLNodes; ++b3)
                        for (int a3 = 0; a3 < kLNodes; ++a3, ++a)
                            P[(size_t)b * kLOut + a] = (float)(wc[c3] * wb[b3] * wa[a3]);
            }
}

int history_t0(const LGeom &g, double cdt)
{
    const double hs = 0.5 * g.h_s * std::sqrt((double)(g.n_s[0] - 1) * (g.n_s[0] - 1) +
                                              (double)(g.n_s[1] - 1) * (g.n_s[1] - 1) +
                                              (double)(g.n_s[2] - 1) * (g.n_s[2] - 1));
    return kLWin / 2 + 2 + (int)std::ceil((canonical_half_width(g.Lt) + hs) / cdt);
}

int max_samples(const LGeom &g, double cdt)
{
    // the last window reaches t0 + samples + kLWin/2 + 1 < kLHistT
    return kLHistT - 2 - history_t0(g, cdt) - kLWin / 2 - 1;
}

// Histories [h0, h0 + nh) of a data set: rows X (fp16) and targets Y.
static cudaError_t make_chunk(const LGeom &geo, Rng &rng, int nh, int samples, double c, double dt, __half *X,
                              float *Xf, float *Y, double *desc, cudaStream_t s)
{
    const double cdt = c * dt;
    const long long N = (long long)geo.n_s[0] * geo.n_s[1] * geo.n_s[2];
    const int t0i = history_t0(geo, cdt);
    std::vector<TrainHist> H(nh);
    std::vector<LPair> lp(nh);
    std::vector<FeatRow> rows((size_t)nh * samples);
    double cn[kLOut][3];
    canonical_nodes(geo.Lt, cn);
    for (int i = 0; i < nh; ++i) {
        TrainHist &T = H[i];
        std::memset(&T, 0, sizeof(T));
        const double ext[3] = {geo.h_s * (geo.n_s[0] - 1), geo.h_s * (geo.n_s[1] - 1), geo.h_s * (geo.n_s[2] - 1)};
        T.csx = (float)(0.5 * ext[0]);
        T.csy = (float)(0.5 * ext[1]);
        T.csz = (float)(0.5 * ext[2]);
        const double tshift = rng.uniform(0.0, 1000.0);
        for (int g = 0; g < kLGauss; ++g) {
            T.cx[g] = (float)rng.uniform(0.25 * ext[0], 0.75 * ext[0]);
            T.cy[g] = (float)rng.uniform(0.25 * ext[1], 0.75 * ext[1]);
            T.cz[g] = (float)rng.uniform(0.25 * ext[2], 0.75 * ext[2]);
            T.sigma[g] = (float)rng.uniform(0.4, 1.2);
            const double a = rng.uniform(0.3, 2.0), e = rng.uniform(0.02, 0.3), w = rng.uniform(0.05, 0.8);
            const double ph = rng.uniform(0.0, 2.0 * M_PI);
            for (int j = 0; j < kLHistT; ++j) {
                const double t = (tshift + j) * dt;
                T.amp[g][j] = (float)(a * (1.0 + e * std::sin(w * t + ph)));
                T.damp[g][j] = (float)(a * e * w * std::cos(w * t + ph) / (4.0 * M_PI));
            }
        }
        // geometry: fixed, or a random direction and a log-uniform distance
        double n[3], Rc;
        if (geo.random) {
            double nn = 0.0;
            do {
                for (double &v : n) v = rng.normal();
                nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            } while (nn < 1e-6);
            for (double &v : n) v /= nn;
            Rc = std::exp(rng.uniform(std::log(geo.R_lo), std::log(geo.R_hi)));
        } else {
            for (int k = 0; k < 3; ++k) n[k] = geo.dir[k];
            Rc = geo.Rc;
        }
        double R[9];
        canonical_frame(n, R);
        for (int k = 0; k < 9; ++k) T.R[k] = (float)R[k];
        // window centre of sample 0: for a fixed geometry the evaluation
        // steps are integers (t0 + tau_c integral); a random geometry also
        // draws the fractional part of its delay
        const double tau_c = Rc / cdt;
        const double t0 = geo.random ? t0i + rng.uniform() : t0i + (std::ceil(tau_c) - tau_c);
        for (int a = 0; a < kLOut; ++a) {
            double D[3];
            for (int k = 0; k < 3; ++k)
                D[k] = Rc * n[k] + (geo.label_nodes && !geo.random
                                        ? geo.label_nodes[a][k]
                                        : R[k] * cn[a][0] + R[3 + k] * cn[a][1] + R[6 + k] * cn[a][2]);
            const double Dn = std::sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
            for (int k = 0; k < 3; ++k) T.D[a][k] = (float)D[k];
            T.Dn[a] = (float)Dn;
            T.base[a] = (float)(t0 + (Rc - Dn) / cdt);
        }
        LPair &P = lp[i];
        std::memset(&P, 0, sizeof(P));
        for (int k = 0; k < 9; ++k) P.R[k] = (float)R[k];
        P.tau_c = tau_c;
        P.Rc = (float)Rc;
        P.mdepth = kLHistT;
        for (int k = 0; k < samples; ++k) rows[(size_t)i * samples + k] = FeatRow{i, t0 + k};
        if (desc) {
            double *d = desc + (size_t)i * kLDesc;
            for (int g = 0; g < kLGauss; ++g) {
                d[4 * g] = T.cx[g]; d[4 * g + 1] = T.cy[g]; d[4 * g + 2] = T.cz[g]; d[4 * g + 3] = T.sigma[g];
            }
            for (int g = 0; g < kLGauss; ++g)
                for (int j = 0; j < kLHistT; ++j) {
                    d[4 * kLGauss + g * kLHistT + j] = T.amp[g][j];
                    d[4 * kLGauss + (kLGauss + g) * kLHistT + j] = T.damp[g][j];
                }
            double *tail = d + 4 * kLGauss + 2 * kLGauss * kLHistT;
            tail[0] = t0;
            for (int k = 0; k < 3; ++k) tail[1 + k] = n[k];
            tail[4] = Rc;
        }
    }
    DevBuf<TrainHist> dH;
    DevBuf<LPair> dP;
    DevBuf<FeatRow> dR;
    DevBuf<float> B, Mb, mom, labels, nu;
    DevBuf<double> part;
    DevBuf<MomentJob> dJ;
    cudaError_t e;
    if ((e = dH.alloc(nh)) || (e = dP.alloc(nh)) || (e = dR.alloc(rows.size())) ||
        (e = B.alloc((size_t)nh * kLGauss * 4 * N)) || (e = Mb.alloc((size_t)nh * kLGauss * 4 * kLMom)) ||
        (e = mom.alloc((size_t)nh * kLHistT * 4 * kLMom)) || (e = labels.alloc((size_t)nh * samples * kLOut * 4)) ||
        (e = nu.alloc((size_t)nh * samples * 4)) ||
        (e = part.alloc((size_t)nh * kLGauss * 4 * geo.n_s[2] * kLMom)) || (e = dJ.alloc((size_t)nh * kLGauss)))
        return e;
    for (int i = 0; i < nh; ++i) lp[i].mom = mom.p + (size_t)i * kLHistT * 4 * kLMom;
    // basis moments: one job per (history, Gaussian), fields (g, grad Phi)
    std::vector<MomentJob> jobs((size_t)nh * kLGauss);
    for (int i = 0; i < nh; ++i)
        for (int g = 0; g < kLGauss; ++g) {
            MomentJob &J = jobs[(size_t)i * kLGauss + g];
            std::memset(&J, 0, sizeof(J));
            const float *b = B.p + ((size_t)i * kLGauss + g) * 4 * N;
            J.rho = b;
            J.J = b + N;
            J.nx = geo.n_s[0]; J.ny = geo.n_s[1]; J.nz = geo.n_s[2];
            J.h = geo.h_s;
            J.ox = -H[i].csx; J.oy = -H[i].csy; J.oz = -H[i].csz;
            J.part = part.p + ((size_t)i * kLGauss + g) * 4 * geo.n_s[2] * kLMom;
            J.out = Mb.p + ((size_t)i * kLGauss + g) * 4 * kLMom;
            J.out_depth = 1;
        }
    if ((e = cudaMemcpyAsync(dH.p, H.data(), nh * sizeof(TrainHist), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(dP.p, lp.data(), nh * sizeof(LPair), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(dR.p, rows.data(), rows.size() * sizeof(FeatRow), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(dJ.p, jobs.data(), jobs.size() * sizeof(MomentJob), cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = launch_train_basis(dH.p, nh, geo.n_s, (float)geo.h_s, B.p, s)) ||
        (e = launch_moments(dJ.p, (int)jobs.size(), geo.n_s[2], 0, nullptr, s)) ||
        (e = launch_train_moments(dH.p, nh, Mb.p, kLHistT, mom.p, s)) ||
        (e = launch_train_labels(dH.p, nh, B.p, geo.n_s, (float)geo.h_s, samples, cdt, labels.p, s)) ||
        (e = launch_features(dP.p, dR.p, (int)rows.size(), 0, X, Xf, nu.p, s)) ||
        (e = launch_label_rows(dH.p, nh, labels.p, nu.p, samples, Y, s)))
        return e;
    return cudaStreamSynchronize(s);   // the chunk's scratch is freed on return
}

cudaError_t learned_dataset(const LGeom &geo, uint64_t seed, int nh, int samples, double c, double dt, __half *X,
                            float *Xf, float *Y, cudaStream_t s, double *desc)
{
    Rng rng{seed};
    const long long N = (long long)geo.n_s[0] * geo.n_s[1] * geo.n_s[2];
    // chunks of histories whose basis fields stay within about 512 MB
    const int chunk = (int)std::max<long long>(1, std::min<long long>(nh, (512LL << 20) / (kLGauss * 16 * N)));
    for (int h0 = 0; h0 < nh; h0 += chunk) {
        const int n = std::min(chunk, nh - h0);
        const size_t r0 = (size_t)h0 * samples * 4;
        cudaError_t e = make_chunk(geo, rng, n, samples, c, dt, X + r0 * kLIn, Xf ? Xf + r0 * kLIn : nullptr,
                                   Y + r0 * kLOut, desc ? desc + (size_t)h0 * kLDesc : nullptr, s);
        if (e) return e;
    }
    return cudaSuccess;
}

cudaError_t learned_train(Mlp &net, const __half *X, const float *Y, int rows, int iterations, int batch, float lr,
                          uint64_t seed, int optin, int sms, cudaStream_t s, float *final_loss)
{
    if (batch > net.cap || batch % 128 || rows <= 0) return cudaErrorInvalidValue;
    Rng rng{seed ^ 0x5DEECE66Dull};
    // all minibatch indices up front (sampling with replacement)
    std::vector<int> idx((size_t)iterations * batch);
    for (int &v : idx) v = (int)(rng.next() % (uint64_t)rows);
    DevBuf<int> d_idx;
    cudaError_t e;
    if ((e = d_idx.alloc(idx.size())) ||
        (e = cudaMemcpyAsync(d_idx.p, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, s)))
        return e;
    for (int it = 0; it < iterations; ++it) {
        // cosine decay to 2% of lr
        const float f = 0.02f + 0.98f * 0.5f * (1.0f + std::cos((float)M_PI * it / std::max(1, iterations - 1)));
        if ((e = mlp_gather(net, X, Y, d_idx.p + (size_t)it * batch, batch, s)) ||
            (e = mlp_forward(net, batch, true, optin, sms, s)) || (e = mlp_backward(net, batch, optin, sms, s)) ||
            (e = mlp_adam(net, batch, lr * f, s)))
            return e;
    }
    if (final_loss) return mlp_loss(net, batch, final_loss, s);
    return cudaStreamSynchronize(s);
}

cudaError_t learned_fit_linear(Mlp &net, const float *Xf, const float *Y, int rows, float *Yres, cudaStream_t s)
{
    DevBuf<double> G, B;
    cudaError_t e;
    if ((e = G.alloc((size_t)kLIn * kLIn)) || (e = B.alloc((size_t)kLIn * kLOut)) ||
        (e = linear_normal(Xf, Y, rows, G.p, B.p, s)))
        return e;
    std::vector<double> A((size_t)kLIn * kLIn), b((size_t)kLIn * kLOut);
    if ((e = cudaMemcpyAsync(A.data(), G.p, A.size() * sizeof(double), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(b.data(), B.p, b.size() * sizeof(double), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return e;
    // ridge-regularised normal equations (A + lambda I) w = b, Cholesky in FP64
    double tr = 0.0;
    for (int i = 0; i < kLIn; ++i) tr += A[(size_t)i * kLIn + i];
    const double lambda = 1e-9 * tr / kLIn + 1e-300;
    for (int i = 0; i < kLIn; ++i) A[(size_t)i * kLIn + i] += lambda;
    for (int j = 0; j < kLIn; ++j) {
        double d = A[(size_t)j * kLIn + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * kLIn + k] * A[(size_t)j * kLIn + k];
        if (!(d > 0.0)) return cudaErrorInvalidValue;
        const double l = std::sqrt(d);
        A[(size_t)j * kLIn + j] = l;
        for (int i = j + 1; i < kLIn; ++i) {
            double v = A[(size_t)i * kLIn + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * kLIn + k] * A[(size_t)j * kLIn + k];
            A[(size_t)i * kLIn + j] = v / l;
        }
    }
    std::vector<float> W((size_t)kLOut * kLIn);
    std::vector<double> z(kLIn);
    for (int o = 0; o < kLOut; ++o) {
        for (int i = 0; i < kLIn; ++i) {          // L z = b
            double v = b[(size_t)i * kLOut + o];
            for (int k = 0; k < i; ++k) v -= A[(size_t)i * kLIn + k] * z[k];
            z[i] = v / A[(size_t)i * kLIn + i];
        }
        for (int i = kLIn - 1; i >= 0; --i) {     // L^T w = z
            double v = z[i];
            for (int k = i + 1; k < kLIn; ++k) v -= A[(size_t)k * kLIn + i] * z[k];
            z[i] = v / A[(size_t)i * kLIn + i];
        }
        for (int i = 0; i < kLIn; ++i) W[(size_t)i * kLOut + o] = (float)z[i];   // stored transposed
    }
    if ((e = cudaMemcpyAsync(net.Wlin, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice, s))) return e;
    if (!Yres) return cudaStreamSynchronize(s);
    // the network's targets: what the skip leaves, Y - Wlin x, scaled to unit RMS
    if ((e = linear_apply(net.Wlin, Xf, rows, Y, -1.0f, Yres, s))) return e;
    std::vector<float> r((size_t)rows * kLOut);
    if ((e = cudaMemcpyAsync(r.data(), Yres, r.size() * sizeof(float), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return e;
    double ss = 0.0;
    for (float v : r) ss += (double)v * v;
    const double rms = std::sqrt(ss / (double)r.size());
    net.out_scale = rms > 0.0 ? (float)rms : 1.0f;
    if ((e = linear_apply(net.Wlin, Xf, rows, Y, -1.0f, Yres, s, 1.0f / net.out_scale))) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t learned_eval(Mlp &net, const __half *X, const float *Xf, const float *Y, int rows, int optin, int sms,
                         cudaStream_t s, double err[4], double err_lin[4], const NodeMap *to_nodes)
{
    std::vector<double> num(4, 0.0), numl(4, 0.0), den(4, 0.0);
    std::vector<int> idx(net.cap);
    std::vector<float> out((size_t)net.cap * kLOut), lin((size_t)net.cap * kLOut), want((size_t)net.cap * kLOut);
    DevBuf<int> d_idx;
    DevBuf<float> d_lin;
    cudaError_t e = d_idx.alloc(net.cap);
    if (!e) e = d_lin.alloc((size_t)net.cap * kLOut);
    if (e) return e;
    for (int r0 = 0; r0 < rows; r0 += net.cap) {
        const int n = std::min(net.cap, rows - r0);
        const int padded = (n + 127) / 128 * 128;
        for (int i = 0; i < padded; ++i) idx[i] = r0 + std::min(i, n - 1);
        if ((e = cudaMemcpyAsync(d_idx.p, idx.data(), padded * sizeof(int), cudaMemcpyHostToDevice, s)) ||
            (e = mlp_gather(net, X, Y, d_idx.p, padded, s)) || (e = mlp_forward(net, padded, false, optin, sms, s)) ||
            (e = linear_apply(net.Wlin, Xf + (size_t)r0 * kLIn, n, nullptr, 1.0f, d_lin.p, s)) ||
            (e = cudaMemcpyAsync(out.data(), net.Z[3], (size_t)n * kLOut * sizeof(float), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(lin.data(), d_lin.p, (size_t)n * kLOut * sizeof(float), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(want.data(), net.Y, (size_t)n * kLOut * sizeof(float), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s)))
            return e;
        std::vector<double> pn(kLOut), pl(kLOut);
        for (int i = 0; i < n; ++i) {
            const int f = (r0 + i) % 4;   // rows are (sample, field) with the field fastest
            for (int a = 0; a < kLOut; ++a) {
                const size_t o = (size_t)i * kLOut + a;
                pn[a] = (double)net.out_scale * out[o] + lin[o];
                pl[a] = lin[o];
            }
            if (to_nodes) {
                std::vector<double> qn(kLOut, 0.0), ql(kLOut, 0.0);
                for (int b = 0; b < kLOut; ++b) {
                    for (int a = 0; a < kLOut; ++a) {
                        const double w = (double)to_nodes->P[(size_t)b * kLOut + a] / to_nodes->Ra[a];
                        qn[b] += w * pn[a];
                        ql[b] += w * pl[a];
                    }
                    qn[b] *= to_nodes->Dn[b];
                    ql[b] *= to_nodes->Dn[b];
                }
                pn.swap(qn);
                pl.swap(ql);
            }
            for (int a = 0; a < kLOut; ++a) {
                const size_t o = (size_t)i * kLOut + a;
                const double w = want[o];
                const double d = pn[a] - w, dl = pl[a] - w;
                num[f] += d * d;
                numl[f] += dl * dl;
                den[f] += w * w;
            }
        }
    }
    for (int f = 0; f < 4; ++f) {
        err[f] = den[f] > 0.0 ? std::sqrt(num[f] / den[f]) : 0.0;
        if (err_lin) err_lin[f] = den[f] > 0.0 ? std::sqrt(numl[f] / den[f]) : 0.0;
    }
    return cudaSuccess;
}

}  // namespace rp
