// Cubical Whitney GYM on a periodic box (Sec. 4): the structured-grid kernel family of the method.
//
// DoFs are the average-normalised cubical Whitney forms (Eq. WhitneyFormDefn): x/y/z edges and faces
// anchored at every vertex (i, j, k), index a * nc + i + nx (j + ny k).  The curl is the finite
// difference of Eq. dIsFiniteDiff with coefficients +-1/h_a; Q1 and M2 are diagonal (lumped masses
// of Eq. YeeMassMatrices, Q1 = Delta_V^-1 I and M2 = Delta_V I by default, or any positive values
// per DoF, e.g. an S(1) SPAI or material weights).  With those the GYM leapfrog
//     x = Q1 e;  b_{n+1/2} = b_{n-1/2} - dt C x;  e_{n+1} = e_n + dt C^T M2 b_{n+1/2}
// is the Yee scheme (Sec. 4, Eq. shearMapsBE).  One step is two kernels, one thread per cell
// updating its three faces, then its three edges; every output is written once, deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/ygm.h"

namespace {

struct YGrid {
    int nx, ny, nz;
    long long nc;
    double ih[3];   // 1 / h
};
__device__ __forceinline__ long long ycell(const YGrid& g, int i, int j, int k) {
    i = i < 0 ? i + g.nx : (i >= g.nx ? i - g.nx : i);
    j = j < 0 ? j + g.ny : (j >= g.ny ? j - g.ny : j);
    k = k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
    return i + (long long)g.nx * (j + (long long)g.ny * k);
}
// b_out = b_in - ctau C (q e) for the three faces of each cell
template <typename real>
__global__ void k_yee_b(YGrid g, const real* __restrict__ e, const real* __restrict__ q, const real* b, real* bo, double ctau) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((long long)g.nx * g.ny));
    const long long n = g.nc;
    auto x = [&](int a, long long cc) { return (double)q[a * n + cc] * (double)e[a * n + cc]; };
    const long long cxp = ycell(g, i + 1, j, k), cyp = ycell(g, i, j + 1, k), czp = ycell(g, i, j, k + 1);
    const double x0 = x(0, c), x1 = x(1, c), x2 = x(2, c);
    // normal x: (1/hy)(x_z(j+1) - x_z) - (1/hz)(x_y(k+1) - x_y)
    const double cx = g.ih[1] * (x(2, cyp) - x2) - g.ih[2] * (x(1, czp) - x1);
    // normal y: (1/hz)(x_x(k+1) - x_x) - (1/hx)(x_z(i+1) - x_z)
    const double cy = g.ih[2] * (x(0, czp) - x0) - g.ih[0] * (x(2, cxp) - x2);
    // normal z: (1/hx)(x_y(i+1) - x_y) - (1/hy)(x_x(j+1) - x_x)
    const double cz = g.ih[0] * (x(1, cxp) - x1) - g.ih[1] * (x(0, cyp) - x0);
    bo[c] = (real)((double)b[c] - ctau * cx);
    bo[n + c] = (real)((double)b[n + c] - ctau * cy);
    bo[2 * n + c] = (real)((double)b[2 * n + c] - ctau * cz);
}
// e += ctau C^T (m b) for the three edges of each cell
template <typename real>
__global__ void k_yee_e(YGrid g, const real* __restrict__ b, const real* __restrict__ m, real* __restrict__ e, double ctau) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((long long)g.nx * g.ny));
    const long long n = g.nc;
    auto y = [&](int a, long long cc) { return (double)m[a * n + cc] * (double)b[a * n + cc]; };
    const long long cxm = ycell(g, i - 1, j, k), cym = ycell(g, i, j - 1, k), czm = ycell(g, i, j, k - 1);
    const double y0 = y(0, c), y1 = y(1, c), y2 = y(2, c);
    const double ex = g.ih[1] * (y2 - y(2, cym)) - g.ih[2] * (y1 - y(1, czm));
    const double ey = g.ih[2] * (y0 - y(0, czm)) - g.ih[0] * (y2 - y(2, cxm));
    const double ez = g.ih[0] * (y1 - y(1, cxm)) - g.ih[1] * (y0 - y(0, cym));
    e[c] = (real)((double)e[c] + ctau * ex);
    e[n + c] = (real)((double)e[n + c] + ctau * ey);
    e[2 * n + c] = (real)((double)e[2 * n + c] + ctau * ez);
}

}  // namespace

struct ygm_yee {
    YGrid g{};
    int precision = YGM_FP64, device = 0;
    size_t rs = 8;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *e = nullptr, *b = nullptr, *q = nullptr, *m = nullptr, *bs = nullptr;   // bs: synchronised read-out
    double tau_cfl = 0.0, dt_prev = 0.0;
    bool staggered = false;
    int64_t step = 0, launches = 0;
    std::string err;
};

static std::string g_yee_err;

#define YCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess) {                                                                   \
            Y->err = std::string(#call) + ": " + cudaGetErrorString(_e);                           \
            return YGM_ECUDA;                                                                      \
        }                                                                                          \
    } while (0)

static int yee_upload(ygm_yee* Y, void** dst, const std::vector<double>& v) {
    YCK(cudaMalloc(dst, v.size() * Y->rs));
    if (Y->precision == YGM_FP64) {
        YCK(cudaMemcpy(*dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(v.begin(), v.end());
        YCK(cudaMemcpy(*dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    }
    return 0;
}

template <typename real>
static void yee_launch_b(ygm_yee* Y, double ctau, void* out) {
    const unsigned blocks = (unsigned)((Y->g.nc + 255) / 256);
    k_yee_b<real><<<blocks, 256, 0, Y->stream>>>(Y->g, (const real*)Y->e, (const real*)Y->q, (const real*)Y->b, (real*)out,
                                                 ctau);
    Y->launches++;
}
template <typename real>
static void yee_launch_e(ygm_yee* Y, double ctau) {
    const unsigned blocks = (unsigned)((Y->g.nc + 255) / 256);
    k_yee_e<real><<<blocks, 256, 0, Y->stream>>>(Y->g, (const real*)Y->b, (const real*)Y->m, (real*)Y->e, ctau);
    Y->launches++;
}
static void yee_b(ygm_yee* Y, double ctau, void* out = nullptr) {
    if (Y->precision == YGM_FP64)
        yee_launch_b<double>(Y, ctau, out ? out : Y->b);
    else
        yee_launch_b<float>(Y, ctau, out ? out : Y->b);
}
static void yee_e(ygm_yee* Y, double ctau) {
    if (Y->precision == YGM_FP64)
        yee_launch_e<double>(Y, ctau);
    else
        yee_launch_e<float>(Y, ctau);
}

extern "C" {

int ygm_yee_create(const int32_t n[3], const double h[3], const double* q1, const double* m2, int32_t precision,
                   int32_t device, void* stream, ygm_yee** out) {
    if (!out) return YGM_EINVAL;
    *out = nullptr;
    if (!n || !h || n[0] < 1 || n[1] < 1 || n[2] < 1 || !(h[0] > 0) || !(h[1] > 0) || !(h[2] > 0)) {
        g_yee_err = "need n >= 1 and h > 0 per axis";
        return YGM_EINVAL;
    }
    if (precision != YGM_FP64 && precision != YGM_FP32) {
        g_yee_err = "precision must be YGM_FP64 or YGM_FP32";
        return YGM_EINVAL;
    }
    ygm_yee* Y = new ygm_yee();
    Y->g.nx = n[0];
    Y->g.ny = n[1];
    Y->g.nz = n[2];
    Y->g.nc = (long long)n[0] * n[1] * n[2];
    for (int a = 0; a < 3; ++a) Y->g.ih[a] = 1.0 / h[a];
    Y->precision = precision;
    Y->rs = precision == YGM_FP64 ? 8 : 4;
    Y->device = device;
    const long long N = 3 * Y->g.nc;
    const double dV = h[0] * h[1] * h[2];
    std::vector<double> qv(N, 1.0 / dV), mv(N, dV);
    for (long long i = 0; i < N; ++i) {
        if (q1) qv[i] = q1[i];
        if (m2) mv[i] = m2[i];
        if (!(qv[i] > 0) || !(mv[i] > 0) || !std::isfinite(qv[i]) || !std::isfinite(mv[i])) {
            delete Y;
            g_yee_err = "Q1 and M2 diagonals must be finite and > 0";
            return YGM_EINVAL;
        }
    }
    // CFL (Prop. stability): omega_max^2 = lambda_max(Q1 C^T M2 C) <= the largest Gershgorin row sum
    // of Q1^1/2 C^T M2 C Q1^1/2 (each face carries 4 edges with |C| = 1/h of its two in-plane axes)
    {
        const YGrid& g = Y->g;
        std::vector<double> row(N, 0.0);
        auto cell = [&](int i, int j, int k) {
            i = (i + g.nx) % g.nx;
            j = (j + g.ny) % g.ny;
            k = (k + g.nz) % g.nz;
            return i + (long long)g.nx * (j + (long long)g.ny * k);
        };
        for (int k = 0; k < g.nz; ++k)
            for (int j = 0; j < g.ny; ++j)
                for (int i = 0; i < g.nx; ++i)
                    for (int a = 0; a < 3; ++a) {
                        // the face with normal a at (i, j, k): edges along p = a+1 and r = a+2
                        const int p = (a + 1) % 3, r = (a + 2) % 3;
                        int op[3] = {0, 0, 0}, orr[3] = {0, 0, 0};
                        op[r] = 1;   // the p-edge shifted along r
                        orr[p] = 1;  // the r-edge shifted along p
                        const long long f = a * g.nc + cell(i, j, k);
                        const long long e4[4] = {p * g.nc + cell(i, j, k), p * g.nc + cell(i + op[0], j + op[1], k + op[2]),
                                                 r * g.nc + cell(i, j, k), r * g.nc + cell(i + orr[0], j + orr[1], k + orr[2])};
                        const double c4[4] = {g.ih[r], g.ih[r], g.ih[p], g.ih[p]};
                        double sum = 0.0;
                        for (int u = 0; u < 4; ++u) sum += c4[u] * std::sqrt(qv[e4[u]]);
                        for (int u = 0; u < 4; ++u) row[e4[u]] += std::sqrt(qv[e4[u]]) * c4[u] * mv[f] * sum;
                    }
        double mx = 0.0;
        for (double v : row) mx = std::max(mx, v);
        Y->tau_cfl = 2.0 / std::sqrt(mx);
    }
    auto bad = [&](int code) {
        g_yee_err = Y->err;
        ygm_yee_destroy(Y);
        return code;
    };
    if (cudaSetDevice(device) != cudaSuccess) {
        Y->err = "cudaSetDevice failed";
        return bad(YGM_ECUDA);
    }
    if (stream) {
        Y->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&Y->stream, cudaStreamNonBlocking) != cudaSuccess) {
            Y->err = "cudaStreamCreate failed";
            return bad(YGM_ECUDA);
        }
        Y->own_stream = true;
    }
    int rc;
    if ((rc = yee_upload(Y, &Y->q, qv)) || (rc = yee_upload(Y, &Y->m, mv))) return bad(rc);
    if (cudaMalloc(&Y->e, N * Y->rs) != cudaSuccess || cudaMalloc(&Y->b, N * Y->rs) != cudaSuccess ||
        cudaMalloc(&Y->bs, N * Y->rs) != cudaSuccess || cudaMemset(Y->e, 0, N * Y->rs) != cudaSuccess ||
        cudaMemset(Y->b, 0, N * Y->rs) != cudaSuccess) {
        Y->err = "device allocation failed";
        return bad(YGM_ENOMEM);
    }
    *out = Y;
    return YGM_OK;
}

int ygm_yee_sizes(const ygm_yee* Y, int64_t* n1, int64_t* n2, double* dt_cfl) {
    if (!Y) return YGM_EINVAL;
    if (n1) *n1 = 3 * Y->g.nc;
    if (n2) *n2 = 3 * Y->g.nc;
    if (dt_cfl) *dt_cfl = Y->tau_cfl;
    return YGM_OK;
}

int ygm_yee_set_state(ygm_yee* Y, const void* e, const void* b, int on_device) {
    if (!Y || !e || !b) return YGM_EINVAL;
    const size_t nb = 3 * Y->g.nc * Y->rs;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    YCK(cudaMemcpyAsync(Y->e, e, nb, kind, Y->stream));
    YCK(cudaMemcpyAsync(Y->b, b, nb, kind, Y->stream));
    if (!on_device) YCK(cudaStreamSynchronize(Y->stream));
    Y->staggered = false;
    Y->step = 0;
    return YGM_OK;
}

int ygm_yee_step(ygm_yee* Y, int64_t n, double dt) {
    if (!Y) return YGM_EINVAL;
    if (n < 0 || !(dt > 0) || !std::isfinite(dt)) {
        Y->err = "need n >= 0 and finite dt > 0";
        return YGM_EINVAL;
    }
    if (dt > Y->tau_cfl * (1.0 + 1e-12)) {
        Y->err = "dt exceeds the (Gershgorin) CFL bound";
        return YGM_ECFL;
    }
    YCK(cudaSetDevice(Y->device));
    if (!Y->staggered) {
        yee_b(Y, -0.5 * dt);                  // b_{-1/2} = b_0 + dt/2 C Q1 e_0 (Eq. YeeLeapfrog)
        Y->staggered = true;
    } else if (dt != Y->dt_prev) {
        yee_b(Y, 0.5 * Y->dt_prev - 0.5 * dt);
    }
    Y->dt_prev = dt;
    for (int64_t s = 0; s < n; ++s) {
        yee_b(Y, dt);
        yee_e(Y, dt);
        Y->step++;
    }
    YCK(cudaGetLastError());
    return YGM_OK;
}

int ygm_yee_get_state(ygm_yee* Y, void* e, void* b, int on_device, int synced) {
    if (!Y) return YGM_EINVAL;
    const size_t nb = 3 * Y->g.nc * Y->rs;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e) YCK(cudaMemcpyAsync(e, Y->e, nb, kind, Y->stream));
    if (b) {
        if (synced && Y->staggered) {
            yee_b(Y, 0.5 * Y->dt_prev, Y->bs);   // b_n = b_{n-1/2} - dt/2 C Q1 e_n (the state is untouched)
            YCK(cudaMemcpyAsync(b, Y->bs, nb, kind, Y->stream));
        } else {
            YCK(cudaMemcpyAsync(b, Y->b, nb, kind, Y->stream));
        }
    }
    YCK(cudaGetLastError());
    if (!on_device) YCK(cudaStreamSynchronize(Y->stream));
    return YGM_OK;
}

const char* ygm_yee_last_error(const ygm_yee* Y) { return Y ? Y->err.c_str() : g_yee_err.c_str(); }

void ygm_yee_destroy(ygm_yee* Y) {
    if (!Y) return;
    if (Y->stream) cudaStreamSynchronize(Y->stream);
    cudaFree(Y->e);
    cudaFree(Y->b);
    cudaFree(Y->q);
    cudaFree(Y->m);
    cudaFree(Y->bs);
    if (Y->own_stream && Y->stream) cudaStreamDestroy(Y->stream);
    delete Y;
}

}  // extern "C"
