// FP64 host set-up of the GYM operators (see builder.h).
//
// Paper passages: Sec. 2 (de Rham complex, mass matrices), Sec. 5 (SPAI, Eq. NormalEqSolve,
// symmetrisation, SPD check), Prop. stability (CFL bound), Sec. 3 (shear maps use Q1, C, M2).
#include "builder.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <stdexcept>
#include <thread>

namespace ygm {

// ============================================================== small utilities
static void parallel_for(int64_t n, int threads, const std::function<void(int64_t, int64_t, int)>& fn) {
    if (threads <= 1 || n < 64) {
        fn(0, n, 0);
        return;
    }
    std::vector<std::thread> pool;
    std::atomic<int64_t> next(0);
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(4096, n / (threads * 16) + 1));
    for (int t = 0; t < threads; ++t) {
        pool.emplace_back([&, t]() {
            for (;;) {
                int64_t b = next.fetch_add(chunk);
                if (b >= n) break;
                fn(b, std::min(n, b + chunk), t);
            }
        });
    }
    for (auto& th : pool) th.join();
}

static int default_threads(int t) {
    if (t > 0) return t;
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 4;
}

// Two-wide double vectors (GCC vector extension: SSE2 on x86-64, NEON on aarch64).
typedef double v2d __attribute__((vector_size(16)));
static inline v2d ld2(const double* p) {
    v2d v;
    std::memcpy(&v, p, sizeof(v));
    return v;
}

// Dense symmetric positive definite solve by Cholesky (in place); returns false if not SPD.
// Row-major storage; the factor L overwrites the lower triangle (row i of L is contiguous).
// The trailing update of each 4-column panel is done in 4 x 4 register tiles of dot products
// over the already factored columns, so each loaded value feeds two FMAs.
static bool cholesky_solve(int m, double* A, double* b, int nrhs) {
    for (int j0 = 0; j0 < m; j0 += 4) {
        const int jb = std::min(4, m - j0);
        // panel update: A(i, j0+c) -= sum_{k < j0} L(i, k) L(j0+c, k), i >= j0
        if (j0 > 0) {
            const double* Lj[4];
            for (int c = 0; c < 4; ++c) Lj[c] = A + (int64_t)(j0 + std::min(c, jb - 1)) * m;
            int i0 = j0;
            for (; i0 + 4 <= m; i0 += 4) {
                const double* Li0 = A + (int64_t)i0 * m;
                const double* Li1 = Li0 + m;
                const double* Li2 = Li1 + m;
                const double* Li3 = Li2 + m;
                // 4 x 4 tile of dot products over k, two k at a time in 2-wide vectors
                v2d c00 = {0, 0}, c01 = c00, c02 = c00, c03 = c00, c10 = c00, c11 = c00, c12 = c00, c13 = c00;
                v2d c20 = c00, c21 = c00, c22 = c00, c23 = c00, c30 = c00, c31 = c00, c32 = c00, c33 = c00;
                int k = 0;
                for (; k + 2 <= j0; k += 2) {
                    const v2d b0 = ld2(Lj[0] + k), b1 = ld2(Lj[1] + k), b2 = ld2(Lj[2] + k), b3 = ld2(Lj[3] + k);
                    const v2d x0 = ld2(Li0 + k), x1 = ld2(Li1 + k), x2 = ld2(Li2 + k), x3 = ld2(Li3 + k);
                    c00 += x0 * b0; c01 += x0 * b1; c02 += x0 * b2; c03 += x0 * b3;
                    c10 += x1 * b0; c11 += x1 * b1; c12 += x1 * b2; c13 += x1 * b3;
                    c20 += x2 * b0; c21 += x2 * b1; c22 += x2 * b2; c23 += x2 * b3;
                    c30 += x3 * b0; c31 += x3 * b1; c32 += x3 * b2; c33 += x3 * b3;
                }
                double acc[4][4] = {{c00[0] + c00[1], c01[0] + c01[1], c02[0] + c02[1], c03[0] + c03[1]},
                                    {c10[0] + c10[1], c11[0] + c11[1], c12[0] + c12[1], c13[0] + c13[1]},
                                    {c20[0] + c20[1], c21[0] + c21[1], c22[0] + c22[1], c23[0] + c23[1]},
                                    {c30[0] + c30[1], c31[0] + c31[1], c32[0] + c32[1], c33[0] + c33[1]}};
                for (; k < j0; ++k) {
                    const double xs[4] = {Li0[k], Li1[k], Li2[k], Li3[k]};
                    for (int r = 0; r < 4; ++r)
                        for (int c = 0; c < 4; ++c) acc[r][c] += xs[r] * Lj[c][k];
                }
                for (int r = 0; r < 4; ++r)
                    for (int c = 0; c < jb; ++c)
                        if (i0 + r >= j0 + c) A[(int64_t)(i0 + r) * m + j0 + c] -= acc[r][c];
            }
            for (; i0 < m; ++i0) {
                const double* Li = A + (int64_t)i0 * m;
                for (int c = 0; c < jb; ++c) {
                    if (i0 < j0 + c) continue;
                    double s = 0;
                    for (int k = 0; k < j0; ++k) s += Li[k] * Lj[c][k];
                    A[(int64_t)i0 * m + j0 + c] -= s;
                }
            }
        }
        // factor the panel columns j0 .. j0+jb-1 (left-looking inside the panel)
        for (int c = 0; c < jb; ++c) {
            const int j = j0 + c;
            double* Aj = A + (int64_t)j * m;
            for (int p = j0; p < j; ++p) Aj[j] -= Aj[p] * Aj[p];
            const double d = Aj[j];
            if (!(d > 0)) return false;
            const double sd = std::sqrt(d);
            Aj[j] = sd;
            const double inv = 1.0 / sd;
            for (int i = j + 1; i < m; ++i) {
                double* Ai = A + (int64_t)i * m;
                double s = Ai[j];
                for (int p = j0; p < j; ++p) s -= Ai[p] * Aj[p];
                Ai[j] = s * inv;
            }
        }
    }
    for (int r = 0; r < nrhs; ++r) {
        double* x = b + (int64_t)r * m;
        for (int i = 0; i < m; ++i) {
            const double* Ai = A + (int64_t)i * m;
            double s = x[i];
            for (int p = 0; p < i; ++p) s -= Ai[p] * x[p];
            x[i] = s / Ai[i];
        }
        for (int i = m - 1; i >= 0; --i) {
            const double* Ai = A + (int64_t)i * m;
            x[i] /= Ai[i];
            const double xi = x[i];
            for (int p = 0; p < i; ++p) x[p] -= Ai[p] * xi;
        }
    }
    return true;
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations (small matrices only).
static void jacobi_eigen(int m, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int i = 0; i < m; ++i)
            for (int j = i + 1; j < m; ++j) off += A[(size_t)i * m + j] * A[(size_t)i * m + j];
        if (off < 1e-30) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                double apq = A[(size_t)p * m + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                double theta = 0.5 * (aqq - app) / apq;
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {
                    double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
                    A[(size_t)k * m + p] = c * akp - s * akq;
                    A[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {
                    double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
                    A[(size_t)p * m + k] = c * apk - s * aqk;
                    A[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
                    V[(size_t)k * m + p] = c * vkp - s * vkq;
                    V[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(m);
    for (int i = 0; i < m; ++i) w[i] = A[(size_t)i * m + i];
}

// ============================================================== lattice
static const int EDGE_D[7] = {1, 2, 3, 4, 5, 6, 7};
static const int FACE_D[12][2] = {{1, 3}, {2, 3}, {1, 5}, {4, 5}, {2, 6}, {4, 6},
                                  {1, 7}, {2, 7}, {3, 7}, {4, 7}, {5, 7}, {6, 7}};
static const int TET_D[6][2] = {{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 6}};
static const int LEDGE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int LFACE[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};

static int face_index(int d1, int d2) {
    for (int i = 0; i < 12; ++i)
        if (FACE_D[i][0] == d1 && FACE_D[i][1] == d2) return i;
    return -1;
}
static inline int bit(int m, int a) { return (m >> a) & 1; }

bool Nbr::operator<(const Nbr& o) const {
    if (d[2] != o.d[2]) return d[2] < o.d[2];
    if (d[1] != o.d[1]) return d[1] < o.d[1];
    if (d[0] != o.d[0]) return d[0] < o.d[0];
    return cls < o.cls;
}
bool Nbr::operator==(const Nbr& o) const {
    return cls == o.cls && d[0] == o.d[0] && d[1] == o.d[1] && d[2] == o.d[2];
}

int64_t Lattice::index(const std::vector<DofClass>& cls, int c, int x, int y, int z) const {
    const Box& b = cls[c].box;
    int r0 = x - b.lo[0], r1 = y - b.lo[1], r2 = z - b.lo[2];
    if (r0 < 0 || r1 < 0 || r2 < 0 || r0 >= b.num[0] || r1 >= b.num[1] || r2 >= b.num[2]) return -1;
    return b.offset + ((int64_t)r2 * b.num[1] + r1) * b.num[0] + r0;
}

void Lattice::build(int n_, int k_, double side) {
    n = n_;
    k = k_;
    h = side / n;
    const int e1 = k, f1 = k * (k - 1), t1 = k * (k - 1) * (k - 2) / 2;
    const int f2 = k * (k + 1) / 2, t2 = (k - 1) * k * (k + 1) / 2;
    auto mk = [&](std::vector<DofClass>& v, int kind, int shape, int j, int ext, bool active) {
        DofClass c{};
        c.kind = kind;
        c.shape = shape;
        c.j = j;
        c.ext = ext;
        c.active = active;
        for (int a = 0; a < 3; ++a) {
            c.box.lo[a] = bit(ext, a) ? 0 : 1;
            c.box.num[a] = bit(ext, a) ? n : n - 1;
        }
        c.box.size = (int64_t)c.box.num[0] * c.box.num[1] * c.box.num[2];
        v.push_back(c);
    };
    c1.clear();
    c2.clear();
    // 1-forms: edge j = 0 Whitney (active), j >= 1 gradients; face: gradient at j = 5 (k = 3)
    for (int s = 0; s < 7; ++s)
        for (int j = 0; j < e1; ++j) mk(c1, 0, s, j, EDGE_D[s], j == 0);
    for (int s = 0; s < 12; ++s)
        for (int j = 0; j < f1; ++j) mk(c1, 1, s, j, FACE_D[s][1], !(k == 3 && j == 5));
    for (int s = 0; s < 6; ++s)
        for (int j = 0; j < t1; ++j) mk(c1, 2, s, j, 7, true);
    // 2-forms: face DoFs are all rows of C; tet DoFs: curls of cell 1-forms (k = 3, j < 3)
    for (int s = 0; s < 12; ++s)
        for (int j = 0; j < f2; ++j) mk(c2, 1, s, j, FACE_D[s][1], true);
    for (int s = 0; s < 6; ++s)
        for (int j = 0; j < t2; ++j) mk(c2, 2, s, j, 7, k == 3 && j < 3);
    int64_t off = 0;
    for (auto& c : c1) {
        c.box.offset = off;
        off += c.box.size;
    }
    N1 = off;
    off = 0;
    for (auto& c : c2) {
        c.box.offset = off;
        off += c.box.size;
    }
    N2 = off;
    n1 = 6 * e1 + 4 * f1 + t1;
    n2 = 4 * f2 + t2;
    // local DoF maps for every tet shape
    for (int s = 0; s < 6; ++s) {
        const int vo[4] = {0, TET_D[s][0], TET_D[s][1], 7};
        loc1[s].clear();
        loc2[s].clear();
        for (int le = 0; le < 6; ++le) {
            int a = LEDGE[le][0], b = LEDGE[le][1];
            int d = vo[b] ^ vo[a];
            for (int j = 0; j < e1; ++j) {
                LocalDof L{(d - 1) * e1 + j, {bit(vo[a], 0), bit(vo[a], 1), bit(vo[a], 2)}};
                loc1[s].push_back(L);
            }
        }
        for (int lf = 0; lf < 4; ++lf) {
            int a = LFACE[lf][0], b = LFACE[lf][1], c = LFACE[lf][2];
            int fs = face_index(vo[b] ^ vo[a], vo[c] ^ vo[a]);
            for (int j = 0; j < f1; ++j) {
                LocalDof L{7 * e1 + fs * f1 + j, {bit(vo[a], 0), bit(vo[a], 1), bit(vo[a], 2)}};
                loc1[s].push_back(L);
            }
            for (int j = 0; j < f2; ++j) {
                LocalDof L{fs * f2 + j, {bit(vo[a], 0), bit(vo[a], 1), bit(vo[a], 2)}};
                loc2[s].push_back(L);
            }
        }
        for (int j = 0; j < t1; ++j) loc1[s].push_back(LocalDof{7 * e1 + 12 * f1 + s * t1 + j, {0, 0, 0}});
        for (int j = 0; j < t2; ++j) loc2[s].push_back(LocalDof{12 * f2 + s * t2 + j, {0, 0, 0}});
    }
    act2.clear();
    for (int r = 0; r < n2; ++r)
        if (c2[loc2[0][r].cls].active) act2.push_back(r);
    n2a = (int)act2.size();
    // incidences: every (shape, local DoF) with class c gives a tet at cube = anchor - off
    inc1.assign(c1.size(), {});
    for (int s = 0; s < 6; ++s)
        for (int r = 0; r < n1; ++r) {
            const LocalDof& L = loc1[s][r];
            inc1[L.cls].push_back(Incidence{{-L.off[0], -L.off[1], -L.off[2]}, s, r});
        }
}

void Lattice::tet_dofs1(int64_t t, int64_t* out) const {
    int s = (int)(t % 6);
    int64_t cube = t / 6;
    int cx = (int)(cube % n), cy = (int)((cube / n) % n), cz = (int)(cube / ((int64_t)n * n));
    for (int r = 0; r < n1; ++r) {
        const LocalDof& L = loc1[s][r];
        out[r] = index1(L.cls, cx + L.off[0], cy + L.off[1], cz + L.off[2]);
    }
}
void Lattice::tet_dofs2(int64_t t, int64_t* out) const {
    int s = (int)(t % 6);
    int64_t cube = t / 6;
    int cx = (int)(cube % n), cy = (int)((cube / n) % n), cz = (int)(cube / ((int64_t)n * n));
    for (int r = 0; r < n2; ++r) {
        const LocalDof& L = loc2[s][r];
        out[r] = index2(L.cls, cx + L.off[0], cy + L.off[1], cz + L.off[2]);
    }
}
void Lattice::decode1(int64_t g, int* cls, int v[3]) const {
    int c = 0;
    while (c + 1 < (int)c1.size() && c1[c + 1].box.offset <= g) ++c;
    const Box& b = c1[c].box;
    int64_t r = g - b.offset;
    v[0] = (int)(r % b.num[0]) + b.lo[0];
    v[1] = (int)((r / b.num[0]) % b.num[1]) + b.lo[1];
    v[2] = (int)(r / ((int64_t)b.num[0] * b.num[1])) + b.lo[2];
    *cls = c;
}

// ============================================================== polynomial bases
// 1-form term: c * l^a * g_m ; 2-form term: c * l^a * (g_p x g_q)
struct T1 {
    double c;
    int a[4];
    int m;
};
struct T2 {
    double c;
    int a[4];
    int p, q;
};
using F1 = std::vector<T1>;
using F2 = std::vector<T2>;
struct Poly {
    std::vector<std::pair<double, std::array<int, 4>>> t;
};
static Poly mono(std::initializer_list<int> idx, double c = 1.0) {
    std::array<int, 4> a{0, 0, 0, 0};
    for (int i : idx) a[i]++;
    Poly P;
    P.t.push_back({c, a});
    return P;
}
static Poly operator+(Poly A, const Poly& B) {
    for (auto& x : B.t) A.t.push_back(x);
    return A;
}
static F1 pw(const Poly& P, int a, int b) {  // P (l_a g_b - l_b g_a)
    F1 f;
    for (auto& [c, al] : P.t) {
        T1 u{c, {al[0], al[1], al[2], al[3]}, b};
        u.a[a]++;
        f.push_back(u);
        T1 v{-c, {al[0], al[1], al[2], al[3]}, a};
        v.a[b]++;
        f.push_back(v);
    }
    return f;
}
static F1 grad(const Poly& P) {
    F1 f;
    for (auto& [c, al] : P.t)
        for (int m = 0; m < 4; ++m)
            if (al[m] > 0) {
                T1 u{c * al[m], {al[0], al[1], al[2], al[3]}, m};
                u.a[m]--;
                f.push_back(u);
            }
    return f;
}
static F2 curl(const F1& f) {
    F2 g;
    for (auto& u : f)
        for (int m = 0; m < 4; ++m)
            if (u.a[m] > 0) {
                T2 v{u.c * u.a[m], {u.a[0], u.a[1], u.a[2], u.a[3]}, m, u.m};
                v.a[m]--;
                g.push_back(v);
            }
    return g;
}
static F2 whitney2(int a, int b, int c) {
    F2 g;
    T2 u{2.0, {0, 0, 0, 0}, b, c};
    u.a[a] = 1;
    g.push_back(u);
    T2 v{2.0, {0, 0, 0, 0}, c, a};
    v.a[b] = 1;
    g.push_back(v);
    T2 w{2.0, {0, 0, 0, 0}, a, b};
    w.a[c] = 1;
    g.push_back(w);
    return g;
}

// Local 1-form basis in the local order of the lattice (edges, faces, cell), plus a flag
// telling which functions are gradients.
static void one_forms(int k, std::vector<F1>& F, std::vector<bool>& is_grad) {
    F.clear();
    is_grad.clear();
    for (int le = 0; le < 6; ++le) {
        int a = LEDGE[le][0], b = LEDGE[le][1];
        F.push_back(pw(mono({}), a, b));
        is_grad.push_back(false);
        if (k >= 2) {
            F.push_back(grad(mono({a, b})));
            is_grad.push_back(true);
        }
        if (k >= 3) {
            F.push_back(grad(mono({a, b, b}) + mono({a, a, b}, -1.0)));
            is_grad.push_back(true);
        }
    }
    for (int lf = 0; lf < 4; ++lf) {
        int a = LFACE[lf][0], b = LFACE[lf][1], c = LFACE[lf][2];
        if (k >= 2) {
            F.push_back(pw(mono({c}), a, b));
            F.push_back(pw(mono({b}), a, c));
            is_grad.push_back(false);
            is_grad.push_back(false);
        }
        if (k >= 3) {
            F.push_back(pw(mono({a, c}), a, b));
            F.push_back(pw(mono({b, c}), a, b));
            F.push_back(pw(mono({a, b}), a, c));
            F.push_back(grad(mono({a, b, c})));
            is_grad.insert(is_grad.end(), {false, false, false, true});
        }
    }
    if (k >= 3) {
        F.push_back(pw(mono({2, 3}), 0, 1));
        F.push_back(pw(mono({1, 3}), 0, 2));
        F.push_back(pw(mono({1, 2}), 0, 3));
        is_grad.insert(is_grad.end(), {false, false, false});
    }
}

static double fact(int n) {
    double r = 1;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}
// int_T l^a dx = 6 |T| a! / (|a| + 3)!
static double bary_integral(const int a[4], double vol) {
    int s = a[0] + a[1] + a[2] + a[3];
    return 6.0 * vol * fact(a[0]) * fact(a[1]) * fact(a[2]) * fact(a[3]) / fact(s + 3);
}
static inline void cross3(const double* u, const double* v, double* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

struct RefTet {
    double X[4][3];
    double g[4][3];
    double vol;
};
static RefTet ref_tet(int s, double h) {
    RefTet R{};
    const int vo[4] = {0, TET_D[s][0], TET_D[s][1], 7};
    for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) R.X[i][a] = h * bit(vo[i], a);
    // gradients of barycentric coordinates: invert [1 x y z]
    double A[4][4];
    for (int i = 0; i < 4; ++i) {
        A[0][i] = 1.0;
        for (int a = 0; a < 3; ++a) A[a + 1][i] = R.X[i][a];
    }
    // Gauss-Jordan inverse of A (4 x 4)
    double M[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) M[i][j] = j < 4 ? A[i][j] : (j - 4 == i ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
        for (int j = 0; j < 8; ++j) std::swap(M[c][j], M[piv][j]);
        double d = M[c][c];
        for (int j = 0; j < 8; ++j) M[c][j] /= d;
        for (int r = 0; r < 4; ++r)
            if (r != c) {
                double f = M[r][c];
                for (int j = 0; j < 8; ++j) M[r][j] -= f * M[c][j];
            }
    }
    // lambda = Ainv [1; x], so grad lambda_i = Ainv[i][1..3]
    for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) R.g[i][a] = M[i][4 + a + 1];
    double e1[3], e2[3], e3[3], cr[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = R.X[1][a] - R.X[0][a];
        e2[a] = R.X[2][a] - R.X[0][a];
        e3[a] = R.X[3][a] - R.X[0][a];
    }
    cross3(e1, e2, cr);
    R.vol = std::fabs(cr[0] * e3[0] + cr[1] * e3[1] + cr[2] * e3[2]) / 6.0;
    return R;
}

static double mass1(const F1& f, const F1& g, const RefTet& R) {
    double s = 0;
    for (auto& u : f)
        for (auto& v : g) {
            int a[4] = {u.a[0] + v.a[0], u.a[1] + v.a[1], u.a[2] + v.a[2], u.a[3] + v.a[3]};
            double dot = R.g[u.m][0] * R.g[v.m][0] + R.g[u.m][1] * R.g[v.m][1] + R.g[u.m][2] * R.g[v.m][2];
            s += u.c * v.c * dot * bary_integral(a, R.vol);
        }
    return s;
}
static double mass2(const F2& f, const F2& g, const RefTet& R) {
    double s = 0;
    for (auto& u : f) {
        double cu[3];
        cross3(R.g[u.p], R.g[u.q], cu);
        for (auto& v : g) {
            double cv[3];
            cross3(R.g[v.p], R.g[v.q], cv);
            int a[4] = {u.a[0] + v.a[0], u.a[1] + v.a[1], u.a[2] + v.a[2], u.a[3] + v.a[3]};
            s += u.c * v.c * (cu[0] * cv[0] + cu[1] * cv[1] + cu[2] * cv[2]) * bary_integral(a, R.vol);
        }
    }
    return s;
}
static void eval1(const F1& f, const double lam[4], const RefTet& R, double out[3]) {
    out[0] = out[1] = out[2] = 0;
    for (auto& u : f) {
        double p = u.c;
        for (int i = 0; i < 4; ++i)
            for (int e = 0; e < u.a[i]; ++e) p *= lam[i];
        for (int a = 0; a < 3; ++a) out[a] += p * R.g[u.m][a];
    }
}

// ============================================================== sparse helpers
double Csr::get(int64_t i, int64_t j) const {
    auto b = col.begin() + ptr[i], e = col.begin() + ptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    if (it != e && *it == j) return val[it - col.begin()];
    return 0.0;
}
void Csr::matvec(const double* x, double* y, int threads) const {
    parallel_for(nrows, threads, [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; ++i) {
            double s = 0;
            for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) s += val[p] * x[col[p]];
            y[i] = s;
        }
    });
}
Csr transpose(const Csr& A) {
    Csr T;
    T.nrows = A.ncols;
    T.ncols = A.nrows;
    T.ptr.assign(T.nrows + 1, 0);
    for (int64_t p = 0; p < (int64_t)A.col.size(); ++p) T.ptr[A.col[p] + 1]++;
    for (int64_t i = 0; i < T.nrows; ++i) T.ptr[i + 1] += T.ptr[i];
    T.col.resize(A.col.size());
    T.val.resize(A.col.size());
    std::vector<int64_t> pos(T.ptr.begin(), T.ptr.end() - 1);
    for (int64_t i = 0; i < A.nrows; ++i)
        for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            int64_t q = pos[A.col[p]]++;
            T.col[q] = i;
            T.val[q] = A.val[p];
        }
    return T;
}
Csr spgemm(const Csr& A, const Csr& B, int threads) {
    Csr C;
    C.nrows = A.nrows;
    C.ncols = B.ncols;
    std::vector<std::vector<int64_t>> rc(A.nrows);
    std::vector<std::vector<double>> rv(A.nrows);
    std::vector<std::vector<double>> acc(threads, std::vector<double>());
    std::vector<std::vector<int64_t>> mark(threads);
    parallel_for(A.nrows, threads, [&](int64_t b, int64_t e, int t) {
        auto& ac = acc[t];
        auto& mk = mark[t];
        if (ac.empty()) {
            ac.assign(B.ncols, 0.0);
            mk.assign(B.ncols, -1);
        }
        std::vector<int64_t> cols;
        for (int64_t i = b; i < e; ++i) {
            cols.clear();
            for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
                int64_t k = A.col[p];
                double a = A.val[p];
                for (int64_t q = B.ptr[k]; q < B.ptr[k + 1]; ++q) {
                    int64_t j = B.col[q];
                    if (mk[j] != i) {
                        mk[j] = i;
                        ac[j] = 0.0;
                        cols.push_back(j);
                    }
                    ac[j] += a * B.val[q];
                }
            }
            std::sort(cols.begin(), cols.end());
            rc[i] = cols;
            rv[i].resize(cols.size());
            for (size_t q = 0; q < cols.size(); ++q) rv[i][q] = ac[cols[q]];
        }
    });
    C.ptr.assign(C.nrows + 1, 0);
    for (int64_t i = 0; i < C.nrows; ++i) C.ptr[i + 1] = C.ptr[i] + (int64_t)rc[i].size();
    C.col.resize(C.ptr.back());
    C.val.resize(C.ptr.back());
    parallel_for(C.nrows, threads, [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; ++i) {
            std::copy(rc[i].begin(), rc[i].end(), C.col.begin() + C.ptr[i]);
            std::copy(rv[i].begin(), rv[i].end(), C.val.begin() + C.ptr[i]);
        }
    });
    return C;
}
static Csr symmetrize(const Csr& A, int threads) {
    // (A + A^T)/2 on the union pattern
    Csr T = transpose(A);
    Csr S;
    S.nrows = A.nrows;
    S.ncols = A.ncols;
    std::vector<std::vector<int64_t>> rc(A.nrows);
    std::vector<std::vector<double>> rv(A.nrows);
    parallel_for(A.nrows, threads, [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; ++i) {
            int64_t p = A.ptr[i], pe = A.ptr[i + 1], q = T.ptr[i], qe = T.ptr[i + 1];
            while (p < pe || q < qe) {
                int64_t cp = p < pe ? A.col[p] : INT64_MAX, cq = q < qe ? T.col[q] : INT64_MAX;
                if (cp == cq) {
                    rc[i].push_back(cp);
                    rv[i].push_back(0.5 * (A.val[p] + T.val[q]));
                    ++p;
                    ++q;
                } else if (cp < cq) {
                    rc[i].push_back(cp);
                    rv[i].push_back(0.5 * A.val[p]);
                    ++p;
                } else {
                    rc[i].push_back(cq);
                    rv[i].push_back(0.5 * T.val[q]);
                    ++q;
                }
            }
        }
    });
    S.ptr.assign(S.nrows + 1, 0);
    for (int64_t i = 0; i < S.nrows; ++i) S.ptr[i + 1] = S.ptr[i] + (int64_t)rc[i].size();
    S.col.resize(S.ptr.back());
    S.val.resize(S.ptr.back());
    for (int64_t i = 0; i < S.nrows; ++i) {
        std::copy(rc[i].begin(), rc[i].end(), S.col.begin() + S.ptr[i]);
        std::copy(rv[i].begin(), rv[i].end(), S.val.begin() + S.ptr[i]);
    }
    return S;
}

// ============================================================== set-up stages
namespace {

struct Builder {
    Setup& S;
    Lattice& L;
    int threads;
    explicit Builder(Setup& s, int th) : S(s), L(s.L), threads(th) {}

    std::vector<F1> F1loc;
    std::vector<bool> isgrad;
    std::vector<std::vector<int32_t>> pat1;   // S(M1) rows (tet sharing)

    int64_t tet_index(int cx, int cy, int cz, int s) const {
        return 6 * ((int64_t)cx + (int64_t)L.n * (cy + (int64_t)L.n * cz)) + s;
    }

    // ---------------------------------------------------------- local blocks
    void local_blocks() {
        const int k = L.k;
        one_forms(k, F1loc, isgrad);
        RefTet R = ref_tet(0, L.h);
        const int n1 = L.n1;
        S.M1loc.assign((size_t)n1 * n1, 0.0);
        for (int i = 0; i < n1; ++i)
            for (int j = 0; j < n1; ++j) S.M1loc[(size_t)i * n1 + j] = mass1(F1loc[i], F1loc[j], R);
        // curl-carrying 2-forms in local 2-form order: per face W2 then curls of the face's
        // non-gradient 1-forms, then curls of the cell 1-forms
        std::vector<F2> F2a;
        std::vector<std::vector<std::pair<int, int>>> crow;  // integer C rows (col, value)
        const int per_f1 = k * (k - 1);
        int le_of[4][4];
        for (int le = 0; le < 6; ++le) {
            le_of[LEDGE[le][0]][LEDGE[le][1]] = le;
        }
        for (int lf = 0; lf < 4; ++lf) {
            int a = LFACE[lf][0], b = LFACE[lf][1], c = LFACE[lf][2];
            F2a.push_back(whitney2(a, b, c));
            // Stokes on the face: circulation of w_e around the oriented boundary
            crow.push_back({{le_of[b][c] * k, 1}, {le_of[a][c] * k, -1}, {le_of[a][b] * k, 1}});
            for (int j = 0; j < per_f1; ++j) {
                int col = 6 * k + lf * per_f1 + j;
                if (isgrad[col]) continue;
                F2a.push_back(curl(F1loc[col]));
                crow.push_back({{col, 1}});
            }
        }
        if (k >= 3)
            for (int j = 0; j < 3; ++j) {
                int col = 6 * k + 4 * per_f1 + j;
                F2a.push_back(curl(F1loc[col]));
                crow.push_back({{col, 1}});
            }
        if ((int)F2a.size() != L.n2a) throw std::runtime_error("internal: 2-form count mismatch");
        const int n2a = L.n2a;
        S.M2aloc.assign((size_t)n2a * n2a, 0.0);
        for (int i = 0; i < n2a; ++i)
            for (int j = 0; j < n2a; ++j) S.M2aloc[(size_t)i * n2a + j] = mass2(F2a[i], F2a[j], R);
        S.Cloc.assign((size_t)n2a * n1, 0);
        for (int r = 0; r < n2a; ++r)
            for (auto& [c, v] : crow[r]) S.Cloc[(size_t)r * n1 + c] = v;
        S.Wloc.assign((size_t)n1 * n2a, 0.0);
        for (int i = 0; i < n1; ++i)
            for (int r = 0; r < n2a; ++r) {
                double s = 0;
                for (int q = 0; q < n2a; ++q) s += S.Cloc[(size_t)q * n1 + i] * S.M2aloc[(size_t)q * n2a + r];
                S.Wloc[(size_t)i * n2a + r] = s;
            }
    }

    // ---------------------------------------------------------- M1(eps), pattern S(M1)
    void assemble_M1() {
        const int64_t N1 = L.N1;
        const int n1 = L.n1;
        std::vector<std::vector<int64_t>> rc(N1);
        std::vector<std::vector<double>> rv(N1);
        parallel_for(N1, threads, [&](int64_t b, int64_t e, int) {
            std::vector<std::pair<int64_t, double>> acc;
            for (int64_t g = b; g < e; ++g) {
                int c, v[3];
                L.decode1(g, &c, v);
                acc.clear();
                for (const Incidence& in : L.inc1[c]) {
                    int cx = v[0] + in.dcube[0], cy = v[1] + in.dcube[1], cz = v[2] + in.dcube[2];
                    int64_t t = tet_index(cx, cy, cz, in.shape);
                    double ept = S.eps[t];
                    for (int r = 0; r < n1; ++r) {
                        const LocalDof& Ld = L.loc1[in.shape][r];
                        int64_t gj = L.index1(Ld.cls, cx + Ld.off[0], cy + Ld.off[1], cz + Ld.off[2]);
                        if (gj < 0) continue;
                        acc.push_back({gj, ept * S.M1loc[(size_t)in.loc * n1 + r]});
                    }
                }
                std::sort(acc.begin(), acc.end(),
                          [](const std::pair<int64_t, double>& x, const std::pair<int64_t, double>& y) {
                              return x.first < y.first;
                          });
                for (size_t p = 0; p < acc.size();) {
                    int64_t j = acc[p].first;
                    double s = 0;
                    while (p < acc.size() && acc[p].first == j) s += acc[p++].second;
                    rc[g].push_back(j);
                    rv[g].push_back(s);
                }
            }
        });
        Csr& M = S.M1;
        M.nrows = M.ncols = N1;
        M.ptr.assign(N1 + 1, 0);
        for (int64_t i = 0; i < N1; ++i) M.ptr[i + 1] = M.ptr[i] + (int64_t)rc[i].size();
        M.col.resize(M.ptr.back());
        M.val.resize(M.ptr.back());
        for (int64_t i = 0; i < N1; ++i) {
            std::copy(rc[i].begin(), rc[i].end(), M.col.begin() + M.ptr[i]);
            std::copy(rv[i].begin(), rv[i].end(), M.val.begin() + M.ptr[i]);
        }
    }

    // structural pattern rows (int32): S(1), S(M1) or S(M1^2)
    void patterns(int kind, std::vector<std::vector<int32_t>>& P) {
        const int64_t N1 = L.N1;
        P.assign(N1, {});
        if (kind == YGM_PAT_DIAG) {
            for (int64_t i = 0; i < N1; ++i) P[i] = {(int32_t)i};
            return;
        }
        std::vector<std::vector<int32_t>> P1(N1);
        for (int64_t i = 0; i < N1; ++i) {
            P1[i].resize(S.M1.ptr[i + 1] - S.M1.ptr[i]);
            for (int64_t p = S.M1.ptr[i]; p < S.M1.ptr[i + 1]; ++p) P1[i][p - S.M1.ptr[i]] = (int32_t)S.M1.col[p];
        }
        if (kind == YGM_PAT_SM1) {
            P = std::move(P1);
            return;
        }
        parallel_for(N1, threads, [&](int64_t b, int64_t e, int) {
            std::vector<int32_t> u;
            for (int64_t i = b; i < e; ++i) {
                u.clear();
                for (int32_t m : P1[i]) u.insert(u.end(), P1[m].begin(), P1[m].end());
                std::sort(u.begin(), u.end());
                u.erase(std::unique(u.begin(), u.end()), u.end());
                P[i] = u;
            }
        });
    }
    static constexpr int YGM_PAT_DIAG = 1, YGM_PAT_SM1 = 2, YGM_PAT_SM1SQ = 3;

    // ---------------------------------------------------------- entity-orthonormalised basis T
    // T is block diagonal over the mesh entities: the DoFs g of one edge, face or cell are
    // replaced by (M1[g,g])^(-1/2) times themselves (symmetric Lowdin orthonormalisation).
    // power = +0.5 gives the inverse map T^-1 (blocks (M1[g,g])^(1/2)).
    Csr ortho_T(double power = -0.5) {
        const int64_t N1 = L.N1;
        const Csr& Mp = S.M1;
        // entity groups: DoFs of the same class kind/shape/anchor; classes of an entity are
        // consecutive in j, so group = all classes with the same (kind, shape) at one anchor
        std::vector<std::vector<int64_t>> groups;
        {
            std::map<std::pair<int, int>, std::vector<int>> ent;  // (kind, shape) -> classes
            for (int c = 0; c < (int)L.c1.size(); ++c) ent[{L.c1[c].kind, L.c1[c].shape}].push_back(c);
            for (auto& [key, cl] : ent) {
                const Box& b0 = L.c1[cl[0]].box;
                for (int64_t r = 0; r < b0.size; ++r) {
                    std::vector<int64_t> g;
                    for (int c : cl) g.push_back(L.c1[c].box.offset + r);
                    groups.push_back(g);
                }
            }
        }
        std::vector<std::vector<std::pair<int64_t, double>>> lrows(N1);
        parallel_for((int64_t)groups.size(), threads, [&](int64_t b, int64_t e, int) {
            std::vector<double> A, w, V;
            for (int64_t gi = b; gi < e; ++gi) {
                auto& g = groups[gi];
                int m = (int)g.size();
                A.assign((size_t)m * m, 0.0);
                for (int a = 0; a < m; ++a)
                    for (int c = 0; c < m; ++c) A[(size_t)a * m + c] = Mp.get(g[a], g[c]);
                jacobi_eigen(m, A, w, V);
                for (int a = 0; a < m; ++a)
                    for (int c = 0; c < m; ++c) {
                        double s = 0;
                        for (int q = 0; q < m; ++q) s += V[(size_t)a * m + q] * V[(size_t)c * m + q] * std::pow(w[q], power);
                        lrows[g[a]].push_back({g[c], s});
                    }
            }
        });
        Csr Lw;
        Lw.nrows = Lw.ncols = N1;
        Lw.ptr.assign(N1 + 1, 0);
        for (int64_t i = 0; i < N1; ++i) {
            std::sort(lrows[i].begin(), lrows[i].end());
            Lw.ptr[i + 1] = Lw.ptr[i] + (int64_t)lrows[i].size();
        }
        for (int64_t i = 0; i < N1; ++i)
            for (auto& [c, v] : lrows[i]) {
                Lw.col.push_back(c);
                Lw.val.push_back(v);
            }
        return Lw;
    }

    // ---------------------------------------------------------- SPAI (Eq. NormalEqSolve)
    // Columns l: q(I_l) = [M(:,I)^T M(:,I)]^-1 M(:,I)^T 1_l with M symmetric, so the normal
    // matrix is accumulated row by row of M(:, I) (only its nonzero rows contribute).
    Csr spai(const Csr& M, const std::vector<std::vector<int32_t>>& P) {
        const int64_t N = M.nrows;
        std::vector<std::vector<double>> qcol(N);
        std::vector<std::vector<int32_t>> markv(threads), rmark(threads);
        std::atomic<bool> fail(false);
        parallel_for(N, threads, [&](int64_t b, int64_t e, int t) {
            auto& mk = markv[t];
            if (mk.empty()) mk.assign(N, -1);
            std::vector<double> G, rhs;
            struct Trip {
                int32_t row;
                int32_t p;
                double v;
            };
            std::vector<Trip> trip, sorted;
            std::vector<int64_t> rowids;
            std::vector<int32_t> cnt, pos;
            for (int64_t l = b; l < e; ++l) {
                const auto& I = P[l];
                const int m = (int)I.size();
                for (int p = 0; p < m; ++p) mk[I[p]] = p;
                G.assign((size_t)m * m, 0.0);
                rhs.assign(m, 0.0);
                // rows r of M(:, I): column I_p of M is row I_p (symmetric).  Group the
                // nonzeros of M(:, I) by row with a marker array, then add each row's outer product.
                auto& rm = rmark[t];
                if (rm.empty()) rm.assign(N, -1);
                rowids.clear();
                trip.clear();
                for (int p = 0; p < m; ++p) {
                    int64_t ip = I[p];
                    for (int64_t q = M.ptr[ip]; q < M.ptr[ip + 1]; ++q) {
                        int64_t r = M.col[q];
                        if (rm[r] < 0) {
                            rm[r] = (int32_t)rowids.size();
                            rowids.push_back(r);
                        }
                        trip.push_back({rm[r], p, M.val[q]});
                    }
                }
                cnt.assign(rowids.size() + 1, 0);
                for (auto& x : trip) cnt[x.row + 1]++;
                for (size_t i = 0; i < rowids.size(); ++i) cnt[i + 1] += cnt[i];
                sorted.resize(trip.size());
                pos.assign(cnt.begin(), cnt.end() - 1);
                for (auto& x : trip) sorted[pos[x.row]++] = x;
                for (size_t rr = 0; rr < rowids.size(); ++rr) {
                    for (int32_t ia = cnt[rr]; ia < cnt[rr + 1]; ++ia) {
                        const int pa = sorted[ia].p;
                        const double va = sorted[ia].v;
                        for (int32_t ib = cnt[rr]; ib < cnt[rr + 1]; ++ib) {
                            const int pb = sorted[ib].p;
                            if (pb <= pa) G[(size_t)pa * m + pb] += va * sorted[ib].v;
                        }
                    }
                }
                for (int64_t r : rowids) rm[r] = -1;
                for (int pa = 0; pa < m; ++pa)
                    for (int pb = pa + 1; pb < m; ++pb) G[(size_t)pa * m + pb] = G[(size_t)pb * m + pa];
                // M(:, I)^T 1_l = M(l, I)
                for (int64_t q = M.ptr[l]; q < M.ptr[l + 1]; ++q) {
                    int64_t c = M.col[q];
                    if (mk[c] >= 0) rhs[mk[c]] = M.val[q];
                }
                if (!cholesky_solve(m, G.data(), rhs.data(), 1)) fail = true;
                qcol[l] = rhs;
                for (int p = 0; p < m; ++p) mk[I[p]] = -1;
            }
        });
        if (fail) throw std::runtime_error("SPAI normal matrix not SPD");
        // Q(i, l) = qcol[l][pos of i in I_l]; build CSR of Q^T (rows = columns l), then symmetrise
        Csr Qt;
        Qt.nrows = Qt.ncols = N;
        Qt.ptr.assign(N + 1, 0);
        for (int64_t l = 0; l < N; ++l) Qt.ptr[l + 1] = Qt.ptr[l] + (int64_t)P[l].size();
        Qt.col.resize(Qt.ptr.back());
        Qt.val.resize(Qt.ptr.back());
        for (int64_t l = 0; l < N; ++l)
            for (size_t p = 0; p < P[l].size(); ++p) {
                Qt.col[Qt.ptr[l] + p] = P[l][p];
                Qt.val[Qt.ptr[l] + p] = qcol[l][p];
            }
        return symmetrize(Qt, threads);
    }

    // ---------------------------------------------------------- P2 = C^T M2 C, row-parallel
    std::vector<double> P2loc;
    void make_P2loc() {
        const int n1 = L.n1, n2a = L.n2a;
        P2loc.assign((size_t)n1 * n1, 0.0);
        for (int i = 0; i < n1; ++i)
            for (int j = 0; j < n1; ++j) {
                double s = 0;
                for (int r = 0; r < n2a; ++r) s += S.Wloc[(size_t)i * n2a + r] * S.Cloc[(size_t)r * n1 + j];
                P2loc[(size_t)i * n1 + j] = s;
            }
    }
    void P2_matvec(const double* x, double* y) {
        const int n1 = L.n1;
        parallel_for(L.N1, threads, [&](int64_t b, int64_t e, int) {
            for (int64_t g = b; g < e; ++g) {
                int c, v[3];
                L.decode1(g, &c, v);
                double s = 0;
                for (const Incidence& in : L.inc1[c]) {
                    int cx = v[0] + in.dcube[0], cy = v[1] + in.dcube[1], cz = v[2] + in.dcube[2];
                    double im = 1.0 / S.mu[tet_index(cx, cy, cz, in.shape)];
                    double t = 0;
                    for (int r = 0; r < n1; ++r) {
                        const LocalDof& Ld = L.loc1[in.shape][r];
                        int64_t gj = L.index1(Ld.cls, cx + Ld.off[0], cy + Ld.off[1], cz + Ld.off[2]);
                        if (gj >= 0) t += P2loc[(size_t)in.loc * n1 + r] * x[gj];
                    }
                    s += im * t;
                }
                y[g] = s;
            }
        });
    }

    // P2 = C^T M2 C assembled as a CSR from the local blocks (needs make_P2loc)
    Csr assemble_P2() {
        const int n1 = L.n1;
        const int64_t N1 = L.N1;
        std::vector<std::vector<int64_t>> rc(N1);
        std::vector<std::vector<double>> rv(N1);
        parallel_for(N1, threads, [&](int64_t b, int64_t e, int) {
            std::vector<std::pair<int64_t, double>> acc;
            for (int64_t g = b; g < e; ++g) {
                int c, v[3];
                L.decode1(g, &c, v);
                acc.clear();
                for (const Incidence& in : L.inc1[c]) {
                    int cx = v[0] + in.dcube[0], cy = v[1] + in.dcube[1], cz = v[2] + in.dcube[2];
                    const double im = 1.0 / S.mu[tet_index(cx, cy, cz, in.shape)];
                    for (int r = 0; r < n1; ++r) {
                        const LocalDof& Ld = L.loc1[in.shape][r];
                        int64_t gj = L.index1(Ld.cls, cx + Ld.off[0], cy + Ld.off[1], cz + Ld.off[2]);
                        if (gj >= 0) acc.push_back({gj, im * P2loc[(size_t)in.loc * n1 + r]});
                    }
                }
                std::sort(acc.begin(), acc.end(),
                          [](const std::pair<int64_t, double>& x, const std::pair<int64_t, double>& y) {
                              return x.first < y.first;
                          });
                for (size_t p = 0; p < acc.size();) {
                    const int64_t j = acc[p].first;
                    double sum = 0;
                    while (p < acc.size() && acc[p].first == j) sum += acc[p++].second;
                    rc[g].push_back(j);
                    rv[g].push_back(sum);
                }
            }
        });
        Csr P;
        P.nrows = P.ncols = N1;
        P.ptr.assign(N1 + 1, 0);
        for (int64_t i = 0; i < N1; ++i) P.ptr[i + 1] = P.ptr[i] + (int64_t)rc[i].size();
        P.col.resize(P.ptr.back());
        P.val.resize(P.ptr.back());
        for (int64_t i = 0; i < N1; ++i) {
            std::copy(rc[i].begin(), rc[i].end(), P.col.begin() + P.ptr[i]);
            std::copy(rv[i].begin(), rv[i].end(), P.val.begin() + P.ptr[i]);
        }
        return P;
    }

    // diagonal of P2 (needs make_P2loc): each incident tet adds its local diagonal entry
    void P2_diag(double* d) {
        const int n1 = L.n1;
        parallel_for(L.N1, threads, [&](int64_t b, int64_t e, int) {
            for (int64_t g = b; g < e; ++g) {
                int c, v[3];
                L.decode1(g, &c, v);
                double s = 0;
                for (const Incidence& in : L.inc1[c]) {
                    int cx = v[0] + in.dcube[0], cy = v[1] + in.dcube[1], cz = v[2] + in.dcube[2];
                    s += P2loc[(size_t)in.loc * n1 + in.loc] / S.mu[tet_index(cx, cy, cz, in.shape)];
                }
                d[g] = s;
            }
        });
    }

    // ---------------------------------------------------------- Lanczos helpers
    // Symmetric Lanczos (three-term recurrence) for op self-adjoint in <x, y> = x^T B y;
    // returns the (smallest, largest) Ritz value.  Extreme Ritz values are found by Sturm
    // bisection on the tridiagonal matrix every 10 steps; the loop stops when both settle.
    static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
        int cnt = 0;
        double q = a[0] - x;
        if (q < 0) ++cnt;
        for (size_t i = 1; i < a.size(); ++i) {
            double d = std::fabs(q) < 1e-300 ? 1e-300 : q;
            q = a[i] - x - b[i - 1] * b[i - 1] / d;
            if (q < 0) ++cnt;
        }
        return cnt;  // number of eigenvalues < x
    }
    static std::pair<double, double> tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b) {
        double lo = a[0], hi = a[0];
        for (size_t i = 0; i < a.size(); ++i) {
            double r = (i > 0 ? std::fabs(b[i - 1]) : 0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0);
            lo = std::min(lo, a[i] - r);
            hi = std::max(hi, a[i] + r);
        }
        const int n = (int)a.size();
        double l = lo, h = hi;
        for (int it = 0; it < 200 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)); ++it) {
            double m = 0.5 * (l + h);
            if (sturm_count(a, b, m) >= 1) h = m; else l = m;
        }
        double emin = 0.5 * (l + h);
        l = lo;
        h = hi;
        for (int it = 0; it < 200 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)); ++it) {
            double m = 0.5 * (l + h);
            if (sturm_count(a, b, m) >= n) h = m; else l = m;
        }
        return {emin, 0.5 * (l + h)};
    }
    std::pair<double, double> lanczos(const std::function<void(const double*, double*)>& op,
                                      const std::function<void(const double*, double*)>& Bop, int iters) {
        const int64_t N = L.N1;
        std::vector<double> v(N), Bv(N), w(N), Bw(N), vp(N, 0.0);
        uint64_t st = 0x12345678ULL;
        for (int64_t i = 0; i < N; ++i) {
            st = st * 6364136223846793005ULL + 1442695040888963407ULL;
            v[i] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        }
        Bop(v.data(), Bv.data());
        double nrm = std::sqrt(std::inner_product(v.begin(), v.end(), Bv.begin(), 0.0));
        for (int64_t i = 0; i < N; ++i) {
            v[i] /= nrm;
            Bv[i] /= nrm;
        }
        std::vector<double> al, be;
        double beta = 0, pmin = 0, pmax = 0;
        std::pair<double, double> ext{0, 0};
        const int m = (int)std::min<int64_t>(iters, N);
        for (int it = 0; it < m; ++it) {
            op(v.data(), w.data());
            for (int64_t i = 0; i < N; ++i) w[i] -= beta * vp[i];
            double a = std::inner_product(w.begin(), w.end(), Bv.begin(), 0.0);
            for (int64_t i = 0; i < N; ++i) w[i] -= a * v[i];
            al.push_back(a);
            Bop(w.data(), Bw.data());
            beta = std::sqrt(std::max(0.0, std::inner_product(w.begin(), w.end(), Bw.begin(), 0.0)));
            if ((it + 1) % 10 == 0 || it + 1 == m || beta <= 1e-300) {
                ext = tridiag_extremes(al, be);
                if (it > 30 && std::fabs(ext.second - pmax) <= 1e-13 * std::fabs(ext.second) &&
                    std::fabs(ext.first - pmin) <= 1e-9 * std::fabs(ext.second))
                    break;
                pmin = ext.first;
                pmax = ext.second;
            }
            if (beta <= 1e-300) break;
            be.push_back(beta);
            for (int64_t i = 0; i < N; ++i) {
                vp[i] = v[i];
                v[i] = w[i] / beta;
                Bv[i] = Bw[i] / beta;
            }
        }
        return ext;
    }

    // ---------------------------------------------------------- stencil tables
    void stencils(int pat) {
        const int nc = (int)L.c1.size();
        std::vector<std::vector<Nbr>> s1(nc), sp(nc);
        for (int c = 0; c < nc; ++c) {
            std::vector<Nbr> u;
            for (const Incidence& in : L.inc1[c])
                for (int r = 0; r < L.n1; ++r) {
                    const LocalDof& Ld = L.loc1[in.shape][r];
                    u.push_back(Nbr{Ld.cls, {in.dcube[0] + Ld.off[0], in.dcube[1] + Ld.off[1], in.dcube[2] + Ld.off[2]}});
                }
            std::sort(u.begin(), u.end());
            u.erase(std::unique(u.begin(), u.end()), u.end());
            s1[c] = u;
        }
        for (int c = 0; c < nc; ++c) {
            if (pat == YGM_PAT_DIAG) {
                sp[c] = {Nbr{c, {0, 0, 0}}};
            } else if (pat == YGM_PAT_SM1) {
                sp[c] = s1[c];
            } else {
                std::vector<Nbr> u;
                for (const Nbr& a : s1[c])
                    for (const Nbr& b : s1[a.cls]) u.push_back(Nbr{b.cls, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}});
                std::sort(u.begin(), u.end());
                u.erase(std::unique(u.begin(), u.end()), u.end());
                sp[c] = u;
            }
        }
        // upper: neighbour at or after (0, c) in the (dz, dy, dx, class) order
        std::vector<std::vector<Nbr>> up(nc);
        for (int c = 0; c < nc; ++c) {
            Nbr self{c, {0, 0, 0}};
            for (const Nbr& a : sp[c])
                if (!(a < self)) up[c].push_back(a);
        }
        S.st_begin.assign(nc + 1, 0);
        S.n_upper.assign(nc, 0);
        S.st_slots.clear();
        for (int c = 0; c < nc; ++c) {
            S.n_upper[c] = (int)up[c].size();
            for (size_t s = 0; s < up[c].size(); ++s) {
                Setup::StencilSlot sl{};
                sl.cls = up[c][s].cls;
                for (int a = 0; a < 3; ++a) sl.d[a] = (int8_t)up[c][s].d[a];
                sl.upper = 1;
                sl.slot = (int)s;
                S.st_slots.push_back(sl);
            }
            Nbr self{c, {0, 0, 0}};
            for (const Nbr& a : sp[c]) {
                if (!(a < self)) continue;
                Nbr back{c, {-a.d[0], -a.d[1], -a.d[2]}};
                auto& U = up[a.cls];
                auto it = std::lower_bound(U.begin(), U.end(), back);
                if (it == U.end() || !(*it == back)) throw std::runtime_error("internal: stencil not symmetric");
                Setup::StencilSlot sl{};
                sl.cls = a.cls;
                for (int q = 0; q < 3; ++q) sl.d[q] = (int8_t)a.d[q];
                sl.upper = 0;
                sl.slot = (int)(it - U.begin());
                S.st_slots.push_back(sl);
            }
            S.st_begin[c + 1] = (int)S.st_slots.size();
        }
        // pack upper values: [class][slot][box index]
        S.qoff.assign(nc + 1, 0);
        for (int c = 0; c < nc; ++c) S.qoff[c + 1] = S.qoff[c] + (int64_t)S.n_upper[c] * L.c1[c].box.size;
        S.qvals.assign(S.qoff[nc], 0.0);
        std::atomic<int64_t> missing(0);
        for (int c = 0; c < nc; ++c) {
            const Box& b = L.c1[c].box;
            parallel_for(b.size, threads, [&](int64_t lo, int64_t hi, int) {
                for (int64_t r = lo; r < hi; ++r) {
                    int v0 = (int)(r % b.num[0]) + b.lo[0];
                    int v1 = (int)((r / b.num[0]) % b.num[1]) + b.lo[1];
                    int v2 = (int)(r / ((int64_t)b.num[0] * b.num[1])) + b.lo[2];
                    int64_t gi = b.offset + r;
                    for (int s = 0; s < S.n_upper[c]; ++s) {
                        const Nbr& a = up[c][s];
                        int64_t gj = L.index1(a.cls, v0 + a.d[0], v1 + a.d[1], v2 + a.d[2]);
                        S.qvals[S.qoff[c] + (int64_t)s * b.size + r] = gj >= 0 ? S.Q1.get(gi, gj) : 0.0;
                    }
                }
            });
        }
        (void)missing;
    }
};

}  // namespace

int build_setup(Setup& S, int n, double side, int k, const double* eps, const double* mu, int q1_pattern,
                int threads_in) {
    const int threads = default_threads(threads_in);
    const bool verbose = std::getenv("YGM_VERBOSE") != nullptr;
    auto tic = std::chrono::steady_clock::now();
    auto stage = [&](const char* what) {
        if (!verbose) return;
        auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[ygm setup] %-28s %8.2f s\n", what, std::chrono::duration<double>(now - tic).count());
        tic = now;
    };
    try {
        S.L.build(n, k, side);
        const int64_t T = 6LL * n * n * n;
        if (eps)
            S.eps.assign(eps, eps + T);
        else
            S.eps.assign(T, 1.0);
        if (mu)
            S.mu.assign(mu, mu + T);
        else
            S.mu.assign(T, 1.0);
        for (int64_t t = 0; t < T; ++t)
            if (!(S.eps[t] > 0) || !(S.mu[t] > 0) || !std::isfinite(S.eps[t]) || !std::isfinite(S.mu[t])) {
                S.err = "eps and mu must be finite and positive";
                return -1;
            }
        Builder B(S, threads);
        B.local_blocks();
        stage("local blocks");
        B.assemble_M1();
        stage("assemble M1");
        int pat = q1_pattern == 0 ? (k == 1 ? Builder::YGM_PAT_SM1 : Builder::YGM_PAT_SM1SQ) : q1_pattern;
        if (pat < 1 || pat > 3) {
            S.err = "unknown q1_pattern";
            return -1;
        }
        S.q1_pattern = pat;
        S.ortho = (k >= 2 && pat == Builder::YGM_PAT_SM1SQ);
        std::vector<std::vector<int32_t>> P;
        B.patterns(pat, P);
        stage("patterns");
        if (S.ortho) {
            Csr Tm = B.ortho_T();
            stage("ortho basis T");
            Csr Mp = spgemm(spgemm(Tm, S.M1, threads), transpose(Tm), threads);
            stage("M' = T M1 T^T");
            Csr Qp = B.spai(Mp, P);
            stage("SPAI columns");
            Csr Q1 = spgemm(spgemm(transpose(Tm), Qp, threads), Tm, threads);
            S.Q1 = symmetrize(Q1, threads);
            stage("Q1 = T^T Q' T");
        } else {
            S.Q1 = B.spai(S.M1, P);
            stage("SPAI columns");
        }
        // SPD check (Sec. 5.1, practical considerations) by Lanczos on Q1
        const int64_t N1 = S.L.N1;
        auto qop = [&](const double* x, double* y) { S.Q1.matvec(x, y, threads); };
        auto idop = [&](const double* x, double* y) { std::copy(x, x + N1, y); };
        auto mm = B.lanczos(qop, idop, 300);
        stage("SPD check (Lanczos)");
        S.lmin = mm.first;
        S.lmax = mm.second;
        S.shift = 0;
        if (S.lmin <= 0) {
            S.shift = std::fabs(S.lmin) + 1e-12 * S.lmax;
            for (int64_t i = 0; i < N1; ++i)
                for (int64_t p = S.Q1.ptr[i]; p < S.Q1.ptr[i + 1]; ++p)
                    if (S.Q1.col[p] == i) S.Q1.val[p] += S.shift;
        }
        // CFL: omega_max^2 = lambda_max(Q1 P2); P2 Q1 is self-adjoint in the Q1 inner product
        B.make_P2loc();
        std::vector<double> tmp(N1);
        auto kop = [&](const double* x, double* y) {
            S.Q1.matvec(x, tmp.data(), threads);
            B.P2_matvec(tmp.data(), y);
        };
        auto cfl = B.lanczos(kop, qop, 400);
        S.omega_max_sq = cfl.second;
        S.tau_cfl = 2.0 / std::sqrt(S.omega_max_sq);
        stage("CFL (Lanczos)");
        B.stencils(pat);
        pack_full(S, threads);
        if (!pack_sym(S, threads)) throw std::runtime_error("internal: 1-form anchor outside the lattice");
        stage("stencils + packing");
    } catch (const std::exception& ex) {
        S.err = ex.what();
        return -3;
    }
    return 0;
}

int refresh_spectrum(Setup& S, int threads_in) {
    const int threads = default_threads(threads_in);
    try {
        Builder B(S, threads);
        const int64_t N1 = S.L.N1;
        auto qop = [&](const double* x, double* y) { S.Q1.matvec(x, y, threads); };
        auto idop = [&](const double* x, double* y) { std::copy(x, x + N1, y); };
        auto mm = B.lanczos(qop, idop, 300);
        S.lmin = mm.first;
        S.lmax = mm.second;
        S.shift = 0;
        if (!(S.lmin > 0)) {
            S.err = "Q1 is not positive definite (Prop. stability needs SPD)";
            return -3;
        }
        B.make_P2loc();
        std::vector<double> tmp(N1);
        auto kop = [&](const double* x, double* y) {
            S.Q1.matvec(x, tmp.data(), threads);
            B.P2_matvec(tmp.data(), y);
        };
        auto cfl = B.lanczos(kop, qop, 400);
        S.omega_max_sq = cfl.second;
        S.tau_cfl = 2.0 / std::sqrt(S.omega_max_sq);
    } catch (const std::exception& ex) {
        S.err = ex.what();
        return -3;
    }
    return 0;
}

// ============================================================== full row storage of Q1
void pack_full(Setup& S, int threads_in) {
    const int threads = default_threads(threads_in);
    const Lattice& L = S.L;
    const size_t nc = L.c1.size();
    S.qf_off.assign(nc + 1, 0);
    S.qf_plane.assign(nc, 0);
    for (size_t c = 0; c < nc; ++c) {
        const Box& b = L.c1[c].box;
        const int64_t plane = ((int64_t)b.num[0] * b.num[1] + 3) / 4 * 4;
        S.qf_plane[c] = plane;
        S.qf_off[c + 1] = S.qf_off[c] + (int64_t)(S.st_begin[c + 1] - S.st_begin[c]) * plane * b.num[2];
    }
    S.qfull.assign(S.qf_off[nc], 0.0);
    for (size_t c = 0; c < nc; ++c) {
        const Box& b = L.c1[c].box;
        const int64_t plane = S.qf_plane[c], ns = S.st_begin[c + 1] - S.st_begin[c];
        parallel_for(b.size, threads, [&](int64_t lo, int64_t hi, int) {
            for (int64_t r = lo; r < hi; ++r) {
                const int rx = (int)(r % b.num[0]), ry = (int)((r / b.num[0]) % b.num[1]);
                const int rz = (int)(r / ((int64_t)b.num[0] * b.num[1]));
                const int v0 = rx + b.lo[0], v1 = ry + b.lo[1], v2 = rz + b.lo[2];
                for (int64_t s = 0; s < ns; ++s) {
                    const auto& st = S.st_slots[S.st_begin[c] + s];
                    const int64_t gj = L.index1(st.cls, v0 + st.d[0], v1 + st.d[1], v2 + st.d[2]);
                    S.qfull[S.qf_off[c] + (s * b.num[2] + rz) * plane + (int64_t)ry * b.num[0] + rx] =
                        gj >= 0 ? S.Q1.get(b.offset + r, gj) : 0.0;
                }
            }
        });
    }
}

// ============================================================== symmetric storage on the anchor lattice
bool pack_sym(Setup& S, int threads_in) {
    const int threads = default_threads(threads_in);
    const Lattice& L = S.L;
    const size_t nc = L.c1.size();
    int H = 0;
    for (const auto& st : S.st_slots)
        for (int a = 0; a < 3; ++a) H = std::max(H, std::abs((int)st.d[a]));
    S.qs_h = H;
    S.qs_nx = (L.n + 7) / 8 * 8;   // rows start on 32-byte boundaries in FP32 and FP64
    S.qs_ny = L.n;
    S.qs_nz = L.n;
    S.qs_vol = (int64_t)S.qs_nx * S.qs_ny * S.qs_nz;
    S.qs_guard = (((int64_t)H * S.qs_ny + H) * S.qs_nx + H + 31) / 32 * 32;
    // the device kernels copy whole runs of 256 lattice points per slot, plus 16 bytes, starting
    // up to 16 bytes below a neighbour address: the band also covers a run that starts at the
    // last lattice point of the last class
    S.qs_guard = std::max<int64_t>(S.qs_guard, 512);
    for (size_t c = 0; c < nc; ++c) {
        const Box& b = L.c1[c].box;
        for (int a = 0; a < 3; ++a)
            if (b.num[a] > 0 && (b.lo[a] < 0 || b.lo[a] + b.num[a] > L.n)) return false;
    }
    S.qs_base.assign(nc + 1, 0);
    S.qs_base[0] = S.qs_guard;
    for (size_t c = 0; c < nc; ++c) S.qs_base[c + 1] = S.qs_base[c] + (int64_t)S.n_upper[c] * S.qs_vol;
    S.qsym.assign(S.qs_base[nc] + S.qs_guard, 0.0);
    for (size_t c = 0; c < nc; ++c) {
        const Box& b = L.c1[c].box;
        const int nup = S.n_upper[c];
        parallel_for(b.size, threads, [&](int64_t lo, int64_t hi, int) {
            for (int64_t r = lo; r < hi; ++r) {
                const int v0 = (int)(r % b.num[0]) + b.lo[0], v1 = (int)((r / b.num[0]) % b.num[1]) + b.lo[1];
                const int v2 = (int)(r / ((int64_t)b.num[0] * b.num[1])) + b.lo[2];
                const int64_t at = ((int64_t)v2 * S.qs_ny + v1) * S.qs_nx + v0;
                for (int s = 0; s < nup; ++s)
                    S.qsym[S.qs_base[c] + s * S.qs_vol + at] = S.qvals[S.qoff[c] + (int64_t)s * b.size + r];
            }
        });
    }
    return true;
}

// ============================================================== user-supplied Q1
int install_q1(Setup& S, const int64_t* rowptr, const int64_t* colind, const double* val, int threads_in) {
    const int threads = default_threads(threads_in);
    const Lattice& L = S.L;
    const int64_t N1 = L.N1;
    // slot lookup per class: (neighbour class, offset) -> present in the stencil
    std::vector<std::map<std::array<int, 4>, int>> slot_of(L.c1.size());
    for (size_t c = 0; c < L.c1.size(); ++c)
        for (int s = S.st_begin[c]; s < S.st_begin[c + 1]; ++s) {
            const auto& st = S.st_slots[s];
            slot_of[c][{st.cls, st.d[0], st.d[1], st.d[2]}] = s;
        }
    Csr Q;
    Q.nrows = Q.ncols = N1;
    Q.ptr.assign(rowptr, rowptr + N1 + 1);
    if (Q.ptr[0] != 0) {
        S.err = "rowptr[0] must be 0";
        return -1;
    }
    for (int64_t i = 0; i < N1; ++i)
        if (Q.ptr[i + 1] < Q.ptr[i]) {
            S.err = "rowptr must be non-decreasing";
            return -1;
        }
    const int64_t nnz = Q.ptr[N1];
    Q.col.assign(colind, colind + nnz);
    Q.val.assign(val, val + nnz);
    double vmax = 0;
    for (int64_t i = 0; i < N1; ++i) {
        int ci, vi[3];
        L.decode1(i, &ci, vi);
        for (int64_t p = Q.ptr[i]; p < Q.ptr[i + 1]; ++p) {
            const int64_t j = Q.col[p];
            if (j < 0 || j >= N1 || (p > Q.ptr[i] && Q.col[p - 1] >= j) || !std::isfinite(Q.val[p])) {
                S.err = "Q1: column indices must be sorted, unique, in range; values finite";
                return -1;
            }
            int cj, vj[3];
            L.decode1(j, &cj, vj);
            if (!slot_of[ci].count({cj, vj[0] - vi[0], vj[1] - vi[1], vj[2] - vi[2]})) {
                S.err = "Q1 has an entry outside the stencil pattern of this context";
                return -1;
            }
            vmax = std::max(vmax, std::fabs(Q.val[p]));
        }
    }
    for (int64_t i = 0; i < N1; ++i)
        for (int64_t p = Q.ptr[i]; p < Q.ptr[i + 1]; ++p)
            if (std::fabs(Q.val[p] - Q.get(Q.col[p], i)) > 1e-14 * vmax) {
                S.err = "Q1 must be symmetric";
                return -1;
            }
    S.Q1 = std::move(Q);
    return repack_q1(S, threads);
}

// Repack the device-facing value tables from S.Q1 and recompute the SPD check and CFL bound.
int repack_q1(Setup& S, int threads_in) {
    const int threads = default_threads(threads_in);
    const Lattice& L = S.L;
    for (size_t c = 0; c < L.c1.size(); ++c) {
        const Box& b = L.c1[c].box;
        parallel_for(b.size, threads, [&](int64_t lo, int64_t hi, int) {
            for (int64_t r = lo; r < hi; ++r) {
                int v0 = (int)(r % b.num[0]) + b.lo[0];
                int v1 = (int)((r / b.num[0]) % b.num[1]) + b.lo[1];
                int v2 = (int)(r / ((int64_t)b.num[0] * b.num[1])) + b.lo[2];
                for (int s = S.st_begin[c]; s < S.st_begin[c + 1]; ++s) {
                    const auto& st = S.st_slots[s];
                    if (!st.upper) continue;
                    int64_t gj = L.index1(st.cls, v0 + st.d[0], v1 + st.d[1], v2 + st.d[2]);
                    S.qvals[S.qoff[c] + (int64_t)st.slot * b.size + r] = gj >= 0 ? S.Q1.get(b.offset + r, gj) : 0.0;
                }
            }
        });
    }
    pack_full(S, threads);
    if (!pack_sym(S, threads)) {
        S.err = "internal: 1-form anchor outside the lattice";
        return -1;
    }
    return refresh_spectrum(S, threads);
}

// ============================================================== SPAI-OP (Sec. 5.1)
// Symmetric Q1 on the pattern of the current Q1 minimising Eq. SPAIOPobjective: the Sylvester
// system (U Q1 T + T Q1 U)_ij = R_ij on the pattern (Eq. SPAIOPSylvester), U = M1^2,
// T = 1 + lam W W^T, W = P2 V, R = M1 T + T M1 (Eq. ThatDefinition), by PCG with the diagonal
// preconditioner of Eq. diagonalPreconditioner, warm-started from the current Q1.  Q1 and U are
// symmetric, so on an entry (i, j):
//   (U Q1 T + T Q1 U)_ij = G_ij + G_ji + lam sum_p (Y_ip W_jp + W_ip Y_jp),  G = U Q1, Y = U Q1 W,
//   R_ij = 2 M1_ij + lam sum_p (Z_ip W_jp + W_ip Z_jp),                       Z = M1 W.
// PCG on the Sylvester system for matrix M, pattern and warm start Q (overwritten with the
// solution, made exactly symmetric), probes W = P2 V (N x np, column-major) in M's basis.
static int sylvester_pcg(const Csr& M, Csr& Q, const std::vector<double>& W, int np, double lam, int maxit,
                         double tol, int threads, int* iters, double* relres, std::string& err) {
    const int64_t N1 = M.nrows;
    const Csr& P = Q;
    const int64_t nq = P.ptr[N1];
    std::vector<double> Z((size_t)N1 * np);
    for (int p = 0; p < np; ++p) M.matvec(&W[(size_t)p * N1], &Z[(size_t)p * N1], threads);
    const Csr U = spgemm(M, M, threads);
    std::vector<int64_t> rowof(nq), tpos(nq);
    for (int64_t i = 0; i < N1; ++i)
        for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) rowof[k] = i;
    for (int64_t k = 0; k < nq; ++k) {
        const int64_t i = rowof[k], j = P.col[k];
        const auto b = P.col.begin() + P.ptr[j], e = P.col.begin() + P.ptr[j + 1];
        const auto it = std::lower_bound(b, e, i);
        if (it == e || *it != i) {
            err = "SPAI-OP: the Q1 pattern is not symmetric";
            return -1;
        }
        tpos[k] = it - P.col.begin();
    }
    std::vector<double> Ud(N1), Td(N1, 1.0);
    for (int64_t i = 0; i < N1; ++i) {
        Ud[i] = U.get(i, i);
        for (int p = 0; p < np; ++p) Td[i] += lam * W[(size_t)p * N1 + i] * W[(size_t)p * N1 + i];
    }
    auto lowrank = [&](const std::vector<double>& Yv, int64_t i, int64_t j) {
        double t = 0;
        for (int p = 0; p < np; ++p)
            t += Yv[(size_t)p * N1 + i] * W[(size_t)p * N1 + j] + W[(size_t)p * N1 + i] * Yv[(size_t)p * N1 + j];
        return lam * t;
    };
    std::vector<double> r(nq), prec(nq);
    for (int64_t k = 0; k < nq; ++k) {
        const int64_t i = rowof[k], j = P.col[k];
        r[k] = 2.0 * M.get(i, j) + (np ? lowrank(Z, i, j) : 0.0);
        prec[k] = Ud[i] * Td[j] + Td[i] * Ud[j];
    }
    // y = A x on the pattern (matrix-free)
    std::vector<double> G(nq), QW((size_t)N1 * np), Y((size_t)N1 * np);
    // one dense column -> slot map per worker thread, reset after every row
    std::vector<std::vector<int64_t>> slots(std::max(1, threads));
    auto apply = [&](const std::vector<double>& x, std::vector<double>& y) {
        // G = U Q (entries of the pattern only), row-parallel
        parallel_for(N1, threads, [&](int64_t b, int64_t e, int th) {
            std::vector<int64_t>& slot = slots[th];
            if (slot.empty()) slot.assign(N1, -1);
            for (int64_t i = b; i < e; ++i) {
                for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) {
                    slot[P.col[k]] = k;
                    G[k] = 0.0;
                }
                for (int64_t a = U.ptr[i]; a < U.ptr[i + 1]; ++a) {
                    const int64_t m = U.col[a];
                    const double u = U.val[a];
                    for (int64_t c = P.ptr[m]; c < P.ptr[m + 1]; ++c) {
                        const int64_t sl = slot[P.col[c]];
                        if (sl >= 0) G[sl] += u * x[c];
                    }
                }
                for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) slot[P.col[k]] = -1;
            }
        });
        if (np > 0) {
            parallel_for(N1, threads, [&](int64_t b, int64_t e, int) {
                for (int64_t i = b; i < e; ++i)
                    for (int p = 0; p < np; ++p) {
                        double t = 0;
                        for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) t += x[k] * W[(size_t)p * N1 + P.col[k]];
                        QW[(size_t)p * N1 + i] = t;
                    }
            });
            for (int p = 0; p < np; ++p) U.matvec(&QW[(size_t)p * N1], &Y[(size_t)p * N1], threads);
        }
        parallel_for(nq, threads, [&](int64_t b, int64_t e, int) {
            for (int64_t k = b; k < e; ++k)
                y[k] = G[k] + G[tpos[k]] + (np ? lowrank(Y, rowof[k], P.col[k]) : 0.0);
        });
    };
    auto dot = [&](const std::vector<double>& a, const std::vector<double>& b2) {
        double t = 0;
        for (int64_t k = 0; k < nq; ++k) t += a[k] * b2[k];
        return t;
    };
    std::vector<double> q(P.val), res(nq), z(nq), pdir(nq), Ap(nq);
    apply(q, Ap);
    for (int64_t k = 0; k < nq; ++k) res[k] = r[k] - Ap[k];
    const double r0 = std::sqrt(dot(r, r));
    double rn = std::sqrt(dot(res, res));
    for (int64_t k = 0; k < nq; ++k) z[k] = res[k] / prec[k];
    pdir = z;
    double rz = dot(res, z);
    int it = 0;
    while (it < maxit && rn > tol * r0) {
        apply(pdir, Ap);
        const double alpha = rz / dot(pdir, Ap);
        for (int64_t k = 0; k < nq; ++k) {
            q[k] += alpha * pdir[k];
            res[k] -= alpha * Ap[k];
        }
        rn = std::sqrt(dot(res, res));
        ++it;
        for (int64_t k = 0; k < nq; ++k) z[k] = res[k] / prec[k];
        const double rz2 = dot(res, z);
        for (int64_t k = 0; k < nq; ++k) pdir[k] = z[k] + (rz2 / rz) * pdir[k];
        rz = rz2;
    }
    if (iters) *iters = it;
    if (relres) *relres = r0 > 0 ? rn / r0 : 0.0;
    if (!(rn <= tol * r0)) {
        err = "SPAI-OP: PCG did not reach the tolerance within max_iter (Q1 unchanged)";
        return -2;
    }
    // the solution is symmetric up to the PCG's rounding (Sec. 5.1); store it exactly so
    for (int64_t k = 0; k < nq; ++k) Q.val[k] = 0.5 * (q[k] + q[tpos[k]]);
    return 0;
}

int spai_op(Setup& S, const double* V, int np, double lam, int maxit, double tol, int threads_in, int* iters,
            double* relres) {
    const int threads = default_threads(threads_in);
    const Lattice& L = S.L;
    const int64_t N1 = L.N1;
    if (np < 0 || (np > 0 && !V) || !(lam >= 0) || !std::isfinite(lam) || maxit < 0 || !(tol > 0)) {
        S.err = "SPAI-OP: need n_probe >= 0 (probe modes when > 0), finite lambda >= 0, max_iter >= 0, tol > 0";
        return -1;
    }
    for (int64_t i = 0; i < N1 * (int64_t)np; ++i)
        if (!std::isfinite(V[i])) {
            S.err = "SPAI-OP: probe modes must be finite";
            return -1;
        }
    try {
        Builder B(S, threads);
        std::vector<double> W((size_t)N1 * np);
        if (np > 0) B.make_P2loc();
        for (int p = 0; p < np; ++p) B.P2_matvec(V + (size_t)p * N1, &W[(size_t)p * N1]);
        int rc;
        if (!S.ortho) {
            Csr Q = S.Q1;
            rc = sylvester_pcg(S.M1, Q, W, np, lam, maxit, tol, threads, iters, relres, S.err);
            if (rc) return rc;
            S.Q1 = std::move(Q);
        } else {
            // orders >= 2: Q1 = T^T Q' T with Q' the SPAI-OP of M' = T M1 T^T in the
            // entity-orthonormal basis, probes W' = T P2 V, warm start Q' = T^-T Q1 T^-1
            const Csr Tm = B.ortho_T(-0.5), Ti = B.ortho_T(0.5);
            const Csr Mp = spgemm(spgemm(Tm, S.M1, threads), transpose(Tm), threads);
            Csr Qp = spgemm(spgemm(transpose(Ti), S.Q1, threads), Ti, threads);
            std::vector<double> Wp((size_t)N1 * np);
            for (int p = 0; p < np; ++p) Tm.matvec(&W[(size_t)p * N1], &Wp[(size_t)p * N1], threads);
            rc = sylvester_pcg(Mp, Qp, Wp, np, lam, maxit, tol, threads, iters, relres, S.err);
            if (rc) return rc;
            Csr Q1 = symmetrize(spgemm(spgemm(transpose(Tm), Qp, threads), Tm, threads), threads);
            if (Q1.ptr != S.Q1.ptr || Q1.col != S.Q1.col) {
                S.err = "internal: SPAI-OP changed the Q1 pattern";
                return -3;
            }
            S.Q1 = std::move(Q1);
        }
    } catch (const std::exception& ex) {
        S.err = ex.what();
        return -3;
    }
    return repack_q1(S, threads);
}

// ============================================================== cavity modes (probe vectors)
// Lowest non-kernel eigenpairs of P2 v = lambda M1 v (the modes of K = M1^-1 P2 that Sec. 5.1 takes
// as SPAI-OP probes).  Block shift-invert subspace iteration in the M1 inner product:
//   Y = (P2 + sigma M1)^-1 M1 X,  Y <- Y minus its M1-projection on ker P2,  M1-orthonormalise Y,
//   Rayleigh-Ritz with Y^T P2 Y,  X = Y Z,
// until every wanted pair has ||P2 x - lambda M1 x|| <= tol lambda ||M1 x||.  ker P2 = ker C is
// spanned by the gradients of the interior vertex hat functions (signed incidence on the Whitney
// edge DoFs; an edge runs from its anchor v to v + d) and by the gradient 1-forms of the
// hierarchical basis (one DoF each).  Inner solves: Jacobi-preconditioned CG.
namespace {
// Jacobi-preconditioned CG for SPD op; returns iterations (or -1 without convergence)
int pcg(const std::function<void(const double*, double*)>& op, const std::vector<double>& dinv, const double* b,
        double* x, int64_t n, double rtol, int maxit) {
    std::vector<double> r(b, b + n), z(n), p(n), q(n);
    std::fill(x, x + n, 0.0);
    double bn = 0;
    for (int64_t i = 0; i < n; ++i) bn += b[i] * b[i];
    bn = std::sqrt(bn);
    if (bn == 0) return 0;
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    p = z;
    double rz = 0;
    for (int64_t i = 0; i < n; ++i) rz += r[i] * z[i];
    for (int it = 1; it <= maxit; ++it) {
        op(p.data(), q.data());
        double pq = 0;
        for (int64_t i = 0; i < n; ++i) pq += p[i] * q[i];
        const double a = rz / pq;
        double rn = 0;
        for (int64_t i = 0; i < n; ++i) {
            x[i] += a * p[i];
            r[i] -= a * q[i];
            rn += r[i] * r[i];
        }
        if (std::sqrt(rn) <= rtol * bn) return it;
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        double rz2 = 0;
        for (int64_t i = 0; i < n; ++i) rz2 += r[i] * z[i];
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + (rz2 / rz) * p[i];
        rz = rz2;
    }
    return -1;
}
}  // namespace

int cavity_modes(Setup& S, int count, double* V, double* lam, int maxit, double tol, int threads_in, int* iters) {
    const Lattice& L = S.L;
    const int64_t N1 = L.N1;
    // the inner loops are light sparse products: worker threads pay off only on large meshes
    const int threads = N1 < 200000 ? 1 : default_threads(threads_in);
    if (count < 1 || !V || !lam || maxit < 1 || !(tol > 0)) {
        S.err = "cavity modes: need count >= 1, output arrays, max_iter >= 1, tol > 0";
        return -1;
    }
    try {
        Builder B(S, threads);
        B.make_P2loc();
        const Csr P2 = B.assemble_P2();
        auto p2mv = [&](const double* a, double* b) { P2.matvec(a, b, threads); };
        // kernel basis as rows of K^T: interior vertex gradients, then the gradient 1-forms
        std::vector<std::vector<std::pair<int64_t, double>>> kt;
        const int n = L.n;
        for (int z = 1; z < n; ++z)
            for (int y = 1; y < n; ++y)
                for (int x = 1; x < n; ++x) {
                    std::vector<std::pair<int64_t, double>> col;
                    for (int c = 0; c < (int)L.c1.size(); ++c) {
                        if (L.c1[c].kind != 0 || L.c1[c].j != 0) continue;
                        const int d = EDGE_D[L.c1[c].shape];
                        const int64_t tail = L.index1(c, x, y, z);                                  // edge x -> x + d
                        const int64_t head = L.index1(c, x - bit(d, 0), y - bit(d, 1), z - bit(d, 2));  // edge x - d -> x
                        if (tail >= 0) col.push_back({tail, -1.0});
                        if (head >= 0) col.push_back({head, 1.0});
                    }
                    std::sort(col.begin(), col.end());
                    kt.push_back(col);
                }
        for (int c = 0; c < (int)L.c1.size(); ++c)
            if (!L.c1[c].active)
                for (int64_t r = 0; r < L.c1[c].box.size; ++r) kt.push_back({{L.c1[c].box.offset + r, 1.0}});
        const int64_t nK = (int64_t)kt.size();
        if (count > N1 - nK) {
            S.err = "cavity modes: count exceeds the number of non-kernel modes";
            return -1;
        }
        Csr Kt;
        Kt.nrows = nK;
        Kt.ncols = N1;
        Kt.ptr.assign(nK + 1, 0);
        for (int64_t i = 0; i < nK; ++i) Kt.ptr[i + 1] = Kt.ptr[i] + (int64_t)kt[i].size();
        for (auto& col : kt)
            for (auto& e : col) {
                Kt.col.push_back(e.first);
                Kt.val.push_back(e.second);
            }
        kt.clear();
        const Csr K = transpose(Kt);
        const Csr L0 = spgemm(spgemm(Kt, S.M1, threads), K, threads);    // K^T M1 K
        std::vector<double> L0inv(nK), Pd(N1), Md(N1), Ainv(N1);
        for (int64_t i = 0; i < nK; ++i) L0inv[i] = 1.0 / L0.get(i, i);
        for (int64_t i = 0; i < N1; ++i) Pd[i] = P2.get(i, i);
        for (int64_t i = 0; i < N1; ++i) Md[i] = S.M1.get(i, i);
        const double sigma = 1.0 / (L.h * L.n * L.h * L.n);               // 1 / side^2
        for (int64_t i = 0; i < N1; ++i) Ainv[i] = 1.0 / (Pd[i] + sigma * Md[i]);
        std::vector<double> t1(N1), t2(N1), kz(nK), kr(nK);
        // self-check: the basis lies in ker P2
        {
            std::vector<double> zz(nK), v(N1), pv(N1);
            for (int64_t i = 0; i < nK; ++i) zz[i] = std::sin(0.37 * (double)i + 0.1);
            K.matvec(zz.data(), v.data(), threads);
            p2mv(v.data(), pv.data());
            double a = 0, bnorm = 0, pmax = 0;
            for (int64_t i = 0; i < N1; ++i) {
                a += pv[i] * pv[i];
                bnorm += v[i] * v[i];
                pmax = std::max(pmax, Pd[i]);
            }
            if (std::sqrt(a) > 1e-10 * pmax * std::sqrt(bnorm)) {
                S.err = "internal: the gradient basis is not in the kernel of P2";
                return -3;
            }
        }
        auto project = [&](double* x) {        // x <- x - K (K^T M1 K)^-1 K^T M1 x
            S.M1.matvec(x, t1.data(), threads);
            Kt.matvec(t1.data(), kr.data(), threads);
            if (pcg([&](const double* a, double* b) { L0.matvec(a, b, threads); }, L0inv, kr.data(), kz.data(), nK,
                    1e-12, 20000) < 0)
                throw std::runtime_error("cavity modes: the kernel projection did not converge");
            K.matvec(kz.data(), t1.data(), threads);
            for (int64_t i = 0; i < N1; ++i) x[i] -= t1[i];
        };
        auto shifted = [&](const double* a, double* b) {   // (P2 + sigma M1) a
            p2mv(a, b);
            S.M1.matvec(a, t2.data(), threads);
            for (int64_t i = 0; i < N1; ++i) b[i] += sigma * t2[i];
        };
        const int p = count + std::max(4, count / 2);
        std::vector<double> X((size_t)N1 * p), Y((size_t)N1 * p), MY((size_t)N1 * p), PY((size_t)N1 * p);
        uint64_t st = 0x9E3779B97F4A7C15ull;                // deterministic start block
        for (auto& v : X) {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            v = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        }
        for (int j = 0; j < p; ++j) project(&X[(size_t)j * N1]);
        std::vector<double> w, Z, H((size_t)p * p);
        int it = 0;
        bool done = false;
        while (it < maxit && !done) {
            ++it;
            for (int j = 0; j < p; ++j) {
                double* y = &Y[(size_t)j * N1];
                S.M1.matvec(&X[(size_t)j * N1], t1.data(), threads);
                std::vector<double> rhs(t1);
                if (pcg(shifted, Ainv, rhs.data(), y, N1, 1e-10, 50000) < 0)
                    throw std::runtime_error("cavity modes: the shifted solve did not converge");
                project(y);
            }
            // M1-orthonormalise Y (Gram-Schmidt, twice)
            for (int pass = 0; pass < 2; ++pass)
                for (int j = 0; j < p; ++j) {
                    double* y = &Y[(size_t)j * N1];
                    for (int i = 0; i < j; ++i) {
                        const double* mi = &MY[(size_t)i * N1];
                        double c = 0;
                        for (int64_t r = 0; r < N1; ++r) c += mi[r] * y[r];
                        const double* yi = &Y[(size_t)i * N1];
                        for (int64_t r = 0; r < N1; ++r) y[r] -= c * yi[r];
                    }
                    double* my = &MY[(size_t)j * N1];
                    S.M1.matvec(y, my, threads);
                    double nn = 0;
                    for (int64_t r = 0; r < N1; ++r) nn += y[r] * my[r];
                    nn = std::sqrt(nn);
                    for (int64_t r = 0; r < N1; ++r) {
                        y[r] /= nn;
                        my[r] /= nn;
                    }
                }
            // Rayleigh-Ritz with P2
            for (int j = 0; j < p; ++j) p2mv(&Y[(size_t)j * N1], &PY[(size_t)j * N1]);
            for (int a = 0; a < p; ++a)
                for (int b2 = 0; b2 < p; ++b2) {
                    double c = 0;
                    for (int64_t r = 0; r < N1; ++r) c += Y[(size_t)a * N1 + r] * PY[(size_t)b2 * N1 + r];
                    H[(size_t)a * p + b2] = c;
                }
            for (int a = 0; a < p; ++a)
                for (int b2 = a + 1; b2 < p; ++b2) H[(size_t)a * p + b2] = H[(size_t)b2 * p + a] =
                    0.5 * (H[(size_t)a * p + b2] + H[(size_t)b2 * p + a]);
            jacobi_eigen(p, H, w, Z);
            std::vector<int> ord(p);
            for (int j = 0; j < p; ++j) ord[j] = j;
            std::sort(ord.begin(), ord.end(), [&](int a, int b2) { return w[a] < w[b2]; });
            double worst = 0;
            for (int jj = 0; jj < p; ++jj) {
                const int j = ord[jj];
                double* x = &X[(size_t)jj * N1];
                std::vector<double> px(N1, 0.0), mx(N1, 0.0);
                for (int a = 0; a < p; ++a) {
                    const double z = Z[(size_t)a * p + j];
                    const double *ya = &Y[(size_t)a * N1], *pa = &PY[(size_t)a * N1], *ma = &MY[(size_t)a * N1];
                    for (int64_t r = 0; r < N1; ++r) {
                        px[r] += z * pa[r];
                        mx[r] += z * ma[r];
                    }
                    if (a == 0)
                        for (int64_t r = 0; r < N1; ++r) x[r] = z * ya[r];
                    else
                        for (int64_t r = 0; r < N1; ++r) x[r] += z * ya[r];
                }
                if (jj < count) {
                    double rn = 0, mn = 0;
                    for (int64_t r = 0; r < N1; ++r) {
                        const double d = px[r] - w[j] * mx[r];
                        rn += d * d;
                        mn += mx[r] * mx[r];
                    }
                    worst = std::max(worst, std::sqrt(rn) / (std::fabs(w[j]) * std::sqrt(mn)));
                    lam[jj] = w[j];
                }
            }
            done = worst <= tol;
        }
        if (iters) *iters = it;
        if (!done) {
            S.err = "cavity modes: not converged within max_iter";
            return -2;
        }
        std::copy(X.begin(), X.begin() + (size_t)count * N1, V);
    } catch (const std::exception& ex) {
        S.err = ex.what();
        return -3;
    }
    return 0;
}

// ============================================================== Q1 vector-Jacobian product in eps
// dL/d eps_T through Q1 (order 1): Q1 = (P + P^T) / 2, P the column SPAI of Eq. NormalEqSolve, so
// with Pbar = (Q1bar + Q1bar^T) / 2 on the pattern, per column l (A = M1(:, I_l), I_l the pattern):
//   q = (A^T A)^-1 A^T 1_l,  r = 1_l - A q,  z = (A^T A)^-1 Pbar(I_l, l),
//   dL/d eps_T += (dA z)^T r - (A z)^T (dA q),   dA = M1^T(:, I_l) (the element matrix of tet T).
// Columns are split into one fixed contiguous range per thread and summed in a fixed order, so the
// result is reproducible for a given thread count.
static int q1_vjp_plain(const Setup& S, const double* q1bar, double* grad, int threads_in) {
    const Lattice& L = S.L;
    const int64_t N1 = L.N1, T = 6LL * L.n * L.n * L.n;
    const Csr& Q = S.Q1;
    const Csr& M = S.M1;
    const int n1 = L.n1;
    // local DoFs of every tet and the tets of every DoF
    std::vector<int64_t> tdofs((size_t)T * n1);
    for (int64_t t = 0; t < T; ++t) L.tet_dofs1(t, &tdofs[(size_t)t * n1]);
    std::vector<int64_t> tptr(N1 + 1, 0), tlist;
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < n1; ++a)
            if (tdofs[(size_t)t * n1 + a] >= 0) ++tptr[tdofs[(size_t)t * n1 + a] + 1];
    for (int64_t i = 0; i < N1; ++i) tptr[i + 1] += tptr[i];
    tlist.resize(tptr[N1]);
    {
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        for (int64_t t = 0; t < T; ++t)
            for (int a = 0; a < n1; ++a) {
                const int64_t g = tdofs[(size_t)t * n1 + a];
                if (g >= 0) tlist[fill[g]++] = t;
            }
    }
    // Pbar on the Q1 pattern (transpose positions by binary search; the pattern is symmetric)
    const int64_t nq = Q.ptr[N1];
    std::vector<double> pbar(nq);
    for (int64_t i = 0; i < N1; ++i)
        for (int64_t k = Q.ptr[i]; k < Q.ptr[i + 1]; ++k) {
            const int64_t j = Q.col[k];
            const auto b = Q.col.begin() + Q.ptr[j], e = Q.col.begin() + Q.ptr[j + 1];
            const auto it = std::lower_bound(b, e, i);
            if (it == e || *it != i) return -1;
            pbar[k] = 0.5 * (q1bar[k] + q1bar[it - Q.col.begin()]);
        }
    const Csr U = spgemm(M, M, 1);     // A^T A = (M1 M1)(I, I) for symmetric M1
    const int threads = std::max(1, std::min<int>(default_threads(threads_in), (int)std::max<int64_t>(1, N1 / 64)));
    std::vector<std::vector<double>> part(threads, std::vector<double>(T, 0.0));
    std::atomic<bool> bad(false);
    auto work = [&](int th) {
        const int64_t l0 = N1 * th / threads, l1 = N1 * (th + 1) / threads;
        std::vector<int32_t> mk(N1, -1);
        std::vector<double> r(N1, 0.0), az(N1, 0.0), G, rhs;
        std::vector<int64_t> rows;
        std::vector<char> rowseen(N1, 0), tseen(T, 0);
        std::vector<int64_t> tets;
        std::vector<double> zT(n1), qT(n1), mz(n1), mq(n1);
        auto& gpart = part[th];
        for (int64_t l = l0; l < l1; ++l) {
            const int64_t* I = &Q.col[Q.ptr[l]];
            const int m = (int)(Q.ptr[l + 1] - Q.ptr[l]);
            for (int p = 0; p < m; ++p) mk[I[p]] = p;
            G.assign((size_t)m * m, 0.0);
            for (int p = 0; p < m; ++p)
                for (int64_t a = U.ptr[I[p]]; a < U.ptr[I[p] + 1]; ++a) {
                    const int32_t pb = mk[U.col[a]];
                    if (pb >= 0) G[(size_t)p * m + pb] = U.val[a];
                }
            rhs.assign((size_t)2 * m, 0.0);
            for (int64_t a = M.ptr[l]; a < M.ptr[l + 1]; ++a)
                if (mk[M.col[a]] >= 0) rhs[mk[M.col[a]]] = M.val[a];
            for (int p = 0; p < m; ++p) rhs[m + p] = pbar[Q.ptr[l] + p];
            if (!cholesky_solve(m, G.data(), rhs.data(), 2)) {
                bad = true;
                break;
            }
            const double* q = rhs.data();
            const double* z = rhs.data() + m;
            // r = 1_l - A q and A z on the rows of A (column I_p of M1 = its row I_p)
            rows.clear();
            for (int p = 0; p < m; ++p)
                for (int64_t a = M.ptr[I[p]]; a < M.ptr[I[p] + 1]; ++a) {
                    const int64_t row = M.col[a];
                    if (!rowseen[row]) {
                        rowseen[row] = 1;
                        rows.push_back(row);
                    }
                    r[row] -= M.val[a] * q[p];
                    az[row] += M.val[a] * z[p];
                }
            r[l] += 1.0;
            // tets holding a DoF of I_l
            tets.clear();
            for (int p = 0; p < m; ++p)
                for (int64_t a = tptr[I[p]]; a < tptr[I[p] + 1]; ++a)
                    if (!tseen[tlist[a]]) {
                        tseen[tlist[a]] = 1;
                        tets.push_back(tlist[a]);
                    }
            std::sort(tets.begin(), tets.end());
            for (int64_t t : tets) {
                const int64_t* D = &tdofs[(size_t)t * n1];
                for (int a = 0; a < n1; ++a) {
                    const int32_t pos = D[a] >= 0 ? mk[D[a]] : -1;
                    zT[a] = pos >= 0 ? z[pos] : 0.0;
                    qT[a] = pos >= 0 ? q[pos] : 0.0;
                }
                double c = 0.0;
                for (int b = 0; b < n1; ++b) {
                    if (D[b] < 0) continue;
                    double sz = 0, sq = 0;
                    for (int a = 0; a < n1; ++a) {
                        sz += S.M1loc[(size_t)b * n1 + a] * zT[a];
                        sq += S.M1loc[(size_t)b * n1 + a] * qT[a];
                    }
                    c += sz * r[D[b]] - az[D[b]] * sq;
                }
                gpart[t] += c;
                tseen[t] = 0;
            }
            for (int64_t row : rows) {
                rowseen[row] = 0;
                r[row] = 0.0;
                az[row] = 0.0;
            }
            r[l] = 0.0;
            for (int p = 0; p < m; ++p) mk[I[p]] = -1;
        }
    };
    std::vector<std::thread> pool;
    for (int th = 0; th < threads; ++th) pool.emplace_back(work, th);
    for (auto& th : pool) th.join();
    if (bad) return -3;
    for (int64_t t = 0; t < T; ++t) {
        double s = 0;
        for (int th = 0; th < threads; ++th) s += part[th][t];
        grad[t] = s;
    }
    return 0;
}

// ---- orders >= 2: Q1 = T Q' T in the entity-orthonormal basis (T = blockdiag M1[g,g]^-1/2)
// Reverse mode (T, Q' symmetric):
//   Q'bar = T Q1bar T, P'bar = (Q'bar + Q'bar^T) / 2 on S,   Tbar  = Q1bar T Q' + Q' T Q1bar
//   column SPAI of M' = T M1 T:  M'bar = sum_l [r z^T - (A z) q^T] in the columns I_l
//   dL/d eps_t += <M'bar, T M1^t T>  (from M1bar = T M'bar T),   Tbar += M'bar T M1 + M1 T M'bar
//   M1bar[g,g] += V (Gamma o (V^T Tbar[g,g] V)) V^T  (A^-1/2 differentiated in the eigenbasis of
//   A = M1[g,g]; Gamma_ij = divided differences of w^-1/2), dL/d eps_t += <M1bar[g,g], M1^t[g,g]>.
// Only the diagonal blocks of Tbar are formed (T is block diagonal), from sparse row dot products
// and per-column accumulations, so no product wider than the Q1 pattern is stored.
static double row_dot(const Csr& A, int64_t i, const Csr& B, int64_t j) {
    int64_t p = A.ptr[i], pe = A.ptr[i + 1], q = B.ptr[j], qe = B.ptr[j + 1];
    double s = 0;
    while (p < pe && q < qe) {
        if (A.col[p] < B.col[q])
            ++p;
        else if (A.col[p] > B.col[q])
            ++q;
        else
            s += A.val[p++] * B.val[q++];
    }
    return s;
}

static int q1_vjp_ortho(Setup& S, const double* q1bar, double* grad, int threads_in) {
    const Lattice& L = S.L;
    const int64_t N1 = L.N1, T = 6LL * L.n * L.n * L.n;
    const int n1 = L.n1;
    const int nthr = default_threads(threads_in);
    Builder B(S, nthr);
    const Csr Tm = B.ortho_T(-0.5), Ti = B.ortho_T(0.5);
    const Csr& Q1 = S.Q1;
    const Csr& M1 = S.M1;
    // groups: the columns of a row of T are the DoFs of its entity
    std::vector<int64_t> gid(N1, -1), gstart;
    std::vector<int64_t> gdofs;
    for (int64_t i = 0; i < N1; ++i) {
        if (gid[i] >= 0) continue;
        const int64_t g = (int64_t)gstart.size();
        gstart.push_back((int64_t)gdofs.size());
        for (int64_t k = Tm.ptr[i]; k < Tm.ptr[i + 1]; ++k) {
            gid[Tm.col[k]] = g;
            gdofs.push_back(Tm.col[k]);
        }
    }
    const int64_t ng = (int64_t)gstart.size();
    gstart.push_back((int64_t)gdofs.size());
    std::vector<int64_t> boff(ng + 1, 0);     // Tbar block storage offsets (|g|^2 each)
    for (int64_t g = 0; g < ng; ++g) {
        const int64_t m = gstart[g + 1] - gstart[g];
        boff[g + 1] = boff[g] + m * m;
    }
    auto gpos = [&](int64_t dof) {         // position of a DoF inside its group
        const int64_t g = gid[dof];
        for (int64_t k = gstart[g]; k < gstart[g + 1]; ++k)
            if (gdofs[k] == dof) return (int)(k - gstart[g]);
        return -1;
    };
    std::vector<int> posv(N1);
    for (int64_t i = 0; i < N1; ++i) posv[i] = gpos(i);
    // Q1bar as a CSR on the Q1 pattern, its transpose, M' = T M1 T, Q' = T^-1 Q1 T^-1, X = T Q'
    Csr Qb = Q1;
    std::copy(q1bar, q1bar + Q1.ptr[N1], Qb.val.begin());
    const Csr QbT = transpose(Qb);
    const Csr Mp = spgemm(spgemm(Tm, M1, nthr), Tm, nthr);
    const Csr Qp = spgemm(spgemm(Ti, Q1, nthr), Ti, nthr);
    const Csr X = spgemm(Tm, Qp, nthr), XT = transpose(X);
    const Csr Y = spgemm(Tm, M1, nthr), YT = transpose(Y);
    const Csr Up = spgemm(Mp, Mp, nthr);
    // P'bar on the pattern of Q' (= S): Q'bar = T Q1bar T, symmetrised
    const Csr QpbarM = spgemm(spgemm(Tm, Qb, nthr), Tm, nthr);
    const int64_t nq = Qp.ptr[N1];
    std::vector<double> pbar(nq);
    for (int64_t i = 0; i < N1; ++i)
        for (int64_t k = Qp.ptr[i]; k < Qp.ptr[i + 1]; ++k) {
            const int64_t j = Qp.col[k];
            pbar[k] = 0.5 * (QpbarM.get(i, j) + QpbarM.get(j, i));
        }
    // Tbar blocks, part 1: Q1bar T Q' + Q' T Q1bar = Q1bar X + X^T Q1bar
    std::vector<double> tbar(boff[ng], 0.0);
    parallel_for(ng, nthr, [&](int64_t g0, int64_t g1, int) {
        for (int64_t g = g0; g < g1; ++g) {
            const int64_t m = gstart[g + 1] - gstart[g];
            for (int64_t a = 0; a < m; ++a)
                for (int64_t b = 0; b < m; ++b) {
                    const int64_t da = gdofs[gstart[g] + a], db = gdofs[gstart[g] + b];
                    tbar[boff[g] + a * m + b] = row_dot(Qb, da, XT, db) + row_dot(XT, da, QbT, db);
                }
        }
    });
    // local DoFs of every tet, the tets of every DoF, and T M1^t T per tet (n1 x n1, local order)
    std::vector<int64_t> tdofs((size_t)T * n1);
    for (int64_t t = 0; t < T; ++t) L.tet_dofs1(t, &tdofs[(size_t)t * n1]);
    std::vector<int64_t> tptr(N1 + 1, 0), tlist;
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < n1; ++a)
            if (tdofs[(size_t)t * n1 + a] >= 0) ++tptr[tdofs[(size_t)t * n1 + a] + 1];
    for (int64_t i = 0; i < N1; ++i) tptr[i + 1] += tptr[i];
    tlist.resize(tptr[N1]);
    {
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        for (int64_t t = 0; t < T; ++t)
            for (int a = 0; a < n1; ++a) {
                const int64_t g = tdofs[(size_t)t * n1 + a];
                if (g >= 0) tlist[fill[g]++] = t;
            }
    }
    std::vector<double> tmt((size_t)T * n1 * n1);
    parallel_for(T, nthr, [&](int64_t t0, int64_t t1, int) {
        std::vector<double> Tl((size_t)n1 * n1), W((size_t)n1 * n1);
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t* D = &tdofs[(size_t)t * n1];
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n1; ++b) Tl[(size_t)a * n1 + b] = (D[a] >= 0 && D[b] >= 0) ? Tm.get(D[a], D[b]) : 0.0;
            for (int a = 0; a < n1; ++a)         // W = Tl Mloc
                for (int b = 0; b < n1; ++b) {
                    double s = 0;
                    for (int c = 0; c < n1; ++c) s += Tl[(size_t)a * n1 + c] * S.M1loc[(size_t)c * n1 + b];
                    W[(size_t)a * n1 + b] = s;
                }
            double* out = &tmt[(size_t)t * n1 * n1];
            for (int a = 0; a < n1; ++a)         // out = W Tl
                for (int b = 0; b < n1; ++b) {
                    double s = 0;
                    for (int c = 0; c < n1; ++c) s += W[(size_t)a * n1 + c] * Tl[(size_t)c * n1 + b];
                    out[(size_t)a * n1 + b] = s;
                }
        }
    });
    // column loop of the SPAI of M' (fixed contiguous ranges per thread, summed in order)
    const int threads = std::max(1, std::min<int>(nthr, (int)std::max<int64_t>(1, N1 / 64)));
    std::vector<std::vector<double>> part(threads, std::vector<double>(T, 0.0));
    std::vector<std::vector<double>> tpart(threads, std::vector<double>(boff[ng], 0.0));
    std::atomic<bool> bad(false);
    auto work = [&](int th) {
        const int64_t l0 = N1 * th / threads, l1 = N1 * (th + 1) / threads;
        std::vector<int32_t> mk(N1, -1);
        std::vector<double> r(N1, 0.0), az(N1, 0.0), wz(N1, 0.0), wq(N1, 0.0), G, rhs;
        std::vector<int64_t> rows, wrows;
        std::vector<char> rowseen(N1, 0), wseen(N1, 0), tseen(T, 0);
        std::vector<int64_t> tets;
        std::vector<double> zT(n1), qT(n1);
        auto& gpart = part[th];
        auto& tb = tpart[th];
        for (int64_t l = l0; l < l1; ++l) {
            const int64_t* I = &Qp.col[Qp.ptr[l]];
            const int m = (int)(Qp.ptr[l + 1] - Qp.ptr[l]);
            for (int p = 0; p < m; ++p) mk[I[p]] = p;
            G.assign((size_t)m * m, 0.0);
            for (int p = 0; p < m; ++p)
                for (int64_t a = Up.ptr[I[p]]; a < Up.ptr[I[p] + 1]; ++a) {
                    const int32_t pb = mk[Up.col[a]];
                    if (pb >= 0) G[(size_t)p * m + pb] = Up.val[a];
                }
            rhs.assign((size_t)2 * m, 0.0);
            for (int64_t a = Mp.ptr[l]; a < Mp.ptr[l + 1]; ++a)
                if (mk[Mp.col[a]] >= 0) rhs[mk[Mp.col[a]]] = Mp.val[a];
            for (int p = 0; p < m; ++p) rhs[m + p] = pbar[Qp.ptr[l] + p];
            if (!cholesky_solve(m, G.data(), rhs.data(), 2)) {
                bad = true;
                break;
            }
            const double* q = rhs.data();
            const double* z = rhs.data() + m;
            rows.clear();
            for (int p = 0; p < m; ++p)
                for (int64_t a = Mp.ptr[I[p]]; a < Mp.ptr[I[p] + 1]; ++a) {
                    const int64_t row = Mp.col[a];
                    if (!rowseen[row]) {
                        rowseen[row] = 1;
                        rows.push_back(row);
                    }
                    r[row] -= Mp.val[a] * q[p];
                    az[row] += Mp.val[a] * z[p];
                }
            if (!rowseen[l]) {
                rowseen[l] = 1;
                rows.push_back(l);
            }
            r[l] += 1.0;
            // (a) <M'bar, T M1^t T> for the tets holding a DoF of I_l
            tets.clear();
            for (int p = 0; p < m; ++p)
                for (int64_t a = tptr[I[p]]; a < tptr[I[p] + 1]; ++a)
                    if (!tseen[tlist[a]]) {
                        tseen[tlist[a]] = 1;
                        tets.push_back(tlist[a]);
                    }
            std::sort(tets.begin(), tets.end());
            for (int64_t t : tets) {
                const int64_t* D = &tdofs[(size_t)t * n1];
                const double* W = &tmt[(size_t)t * n1 * n1];
                for (int a = 0; a < n1; ++a) {
                    const int32_t pos = D[a] >= 0 ? mk[D[a]] : -1;
                    zT[a] = pos >= 0 ? z[pos] : 0.0;
                    qT[a] = pos >= 0 ? q[pos] : 0.0;
                }
                double c = 0.0;
                for (int b = 0; b < n1; ++b) {
                    if (D[b] < 0) continue;
                    double sz = 0, sq = 0;
                    for (int a = 0; a < n1; ++a) {
                        sz += W[(size_t)b * n1 + a] * zT[a];
                        sq += W[(size_t)b * n1 + a] * qT[a];
                    }
                    c += sz * r[D[b]] - az[D[b]] * sq;
                }
                gpart[t] += c;
                tseen[t] = 0;
            }
            // (b) Tbar += M'bar T M1 + M1 T M'bar on the diagonal blocks, Y = T M1:
            //   (M'bar Y)[a,b]   = r_a wz_b - az_a wq_b,  wz = sum_p z_p Y[I_p,:], wq likewise
            //   (Y^T M'bar)[a,b] = z_p (Y^T r)_a - q_p (Y^T az)_a  for b = I_p
            wrows.clear();
            for (int p = 0; p < m; ++p)
                for (int64_t a = Y.ptr[I[p]]; a < Y.ptr[I[p] + 1]; ++a) {
                    const int64_t c = Y.col[a];
                    if (!wseen[c]) {
                        wseen[c] = 1;
                        wrows.push_back(c);
                    }
                    wz[c] += z[p] * Y.val[a];
                    wq[c] += q[p] * Y.val[a];
                }
            for (int64_t a : rows) {
                const int64_t g = gid[a];
                const int64_t mg = gstart[g + 1] - gstart[g];
                const int pa = posv[a];
                for (int64_t bb = 0; bb < mg; ++bb) {
                    const int64_t b = gdofs[gstart[g] + bb];
                    tb[boff[g] + pa * mg + bb] += r[a] * wz[b] - az[a] * wq[b];
                }
            }
            for (int p = 0; p < m; ++p) {
                const int64_t b = I[p];
                const int64_t g = gid[b];
                const int64_t mg = gstart[g + 1] - gstart[g];
                const int pb = posv[b];
                for (int64_t aa = 0; aa < mg; ++aa) {
                    const int64_t a = gdofs[gstart[g] + aa];
                    double yr = 0, ya = 0;         // (Y^T r)_a, (Y^T az)_a: row a of Y^T against dense r, az
                    for (int64_t k = YT.ptr[a]; k < YT.ptr[a + 1]; ++k) {
                        yr += YT.val[k] * r[YT.col[k]];
                        ya += YT.val[k] * az[YT.col[k]];
                    }
                    tb[boff[g] + aa * mg + pb] += z[p] * yr - q[p] * ya;
                }
            }
            for (int64_t c : wrows) {
                wseen[c] = 0;
                wz[c] = 0.0;
                wq[c] = 0.0;
            }
            for (int64_t row : rows) {
                rowseen[row] = 0;
                r[row] = 0.0;
                az[row] = 0.0;
            }
            for (int p = 0; p < m; ++p) mk[I[p]] = -1;
        }
    };
    std::vector<std::thread> pool;
    for (int th = 0; th < threads; ++th) pool.emplace_back(work, th);
    for (auto& th : pool) th.join();
    if (bad) return -3;
    for (int th = 0; th < threads; ++th)
        for (size_t k = 0; k < tbar.size(); ++k) tbar[k] += tpart[th][k];
    for (int64_t t = 0; t < T; ++t) {
        double s = 0;
        for (int th = 0; th < threads; ++th) s += part[th][t];
        grad[t] = s;
    }
    // T = blockdiag f(M1[g,g]), f(w) = w^-1/2: M1bar[g,g] = V (Gamma o (V^T Tbar V)) V^T, then
    // dL/d eps_t += <M1bar[g,g], M1^t[g,g]> for the tets t holding the entity g
    for (int64_t g = 0; g < ng; ++g) {
        const int m = (int)(gstart[g + 1] - gstart[g]);
        const int64_t* gd = &gdofs[gstart[g]];
        std::vector<double> A((size_t)m * m), w, V, C((size_t)m * m), Dm((size_t)m * m);
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) A[(size_t)a * m + b] = M1.get(gd[a], gd[b]);
        jacobi_eigen(m, A, w, V);
        double wmax = 0;
        for (double x : w) wmax = std::max(wmax, std::fabs(x));
        for (int i = 0; i < m; ++i)            // C = V^T Tbar V
            for (int j = 0; j < m; ++j) {
                double s = 0;
                for (int a = 0; a < m; ++a)
                    for (int b = 0; b < m; ++b)
                        s += V[(size_t)a * m + i] * tbar[boff[g] + (int64_t)a * m + b] * V[(size_t)b * m + j];
                const double dw = w[i] - w[j];
                const double gam = std::fabs(dw) <= 1e-12 * wmax ? -0.5 * std::pow(w[i], -1.5)
                                                                 : (std::pow(w[i], -0.5) - std::pow(w[j], -0.5)) / dw;
                C[(size_t)i * m + j] = gam * s;
            }
        for (int a = 0; a < m; ++a)            // Dm = V C V^T
            for (int b = 0; b < m; ++b) {
                double s = 0;
                for (int i = 0; i < m; ++i)
                    for (int j = 0; j < m; ++j) s += V[(size_t)a * m + i] * C[(size_t)i * m + j] * V[(size_t)b * m + j];
                Dm[(size_t)a * m + b] = s;
            }
        for (int64_t k = tptr[gd[0]]; k < tptr[gd[0] + 1]; ++k) {
            const int64_t t = tlist[k];
            const int64_t* D = &tdofs[(size_t)t * n1];
            std::vector<int> loc(m, -1);
            for (int a = 0; a < m; ++a)
                for (int c = 0; c < n1; ++c)
                    if (D[c] == gd[a]) loc[a] = c;
            double s = 0;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) s += Dm[(size_t)a * m + b] * S.M1loc[(size_t)loc[a] * n1 + loc[b]];
            grad[t] += s;
        }
    }
    return 0;
}

int q1_vjp(Setup& S, const double* q1bar, double* grad, int threads) {
    return S.ortho ? q1_vjp_ortho(S, q1bar, grad, threads) : q1_vjp_plain(S, q1bar, grad, threads);
}

// ============================================================== sources and projections
// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n (Golub-Welsch not needed
// for the small orders used here).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (z * p1 - p0) / (z * z - 1);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // refresh derivative at the converged node for the weight
                p0 = 1;
                p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1);
                x[n - 1 - i] = z;
                w[n - 1 - i] = 2.0 / ((1 - z * z) * dp * dp);
                break;
            }
        }
    }
}
static int locate(const Lattice& L, const double x[3], int cube[3], int* shape, double lam[4]) {
    double r[3];
    for (int a = 0; a < 3; ++a) {
        double u = x[a] / L.h;
        int c = (int)std::floor(u);
        c = std::max(0, std::min(L.n - 1, c));
        cube[a] = c;
        r[a] = u - c;
    }
    for (int s = 0; s < 6; ++s) {
        int a1 = TET_D[s][0] == 1 ? 0 : (TET_D[s][0] == 2 ? 1 : 2);
        int d21 = TET_D[s][1] ^ TET_D[s][0];
        int a2 = d21 == 1 ? 0 : (d21 == 2 ? 1 : 2);
        int a3 = 3 - a1 - a2;
        if (r[a1] >= r[a2] - 1e-14 && r[a2] >= r[a3] - 1e-14) {
            *shape = s;
            // barycentric coordinates along the chain: l0 = 1 - r1, l1 = r1 - r2, l2 = r2 - r3, l3 = r3
            lam[0] = 1.0 - r[a1];
            lam[1] = r[a1] - r[a2];
            lam[2] = r[a2] - r[a3];
            lam[3] = r[a3];
            return 0;
        }
    }
    return -1;
}

int dipole_weights(const Setup& S, const double x[3], const double d[3], std::vector<int64_t>& dofs,
                   std::vector<double>& w) {
    const Lattice& L = S.L;
    int cube[3], shape;
    double lam[4];
    if (locate(L, x, cube, &shape, lam)) return -1;
    std::vector<F1> F;
    std::vector<bool> ig;
    one_forms(L.k, F, ig);
    RefTet R = ref_tet(shape, L.h);
    int64_t t = 6 * ((int64_t)cube[0] + (int64_t)L.n * (cube[1] + (int64_t)L.n * cube[2])) + shape;
    std::vector<int64_t> g(L.n1);
    L.tet_dofs1(t, g.data());
    dofs.clear();
    w.clear();
    for (int r = 0; r < L.n1; ++r) {
        if (g[r] < 0) continue;
        double v[3];
        eval1(F[r], lam, R, v);
        dofs.push_back(g[r]);
        w.push_back(v[0] * d[0] + v[1] * d[1] + v[2] * d[2]);
    }
    return 0;
}

int project_E(const Setup& S, void (*E0)(const double*, double*, void*), void* user, std::vector<double>& e0,
              int threads_in) {
    const Lattice& L = S.L;
    const int64_t N1 = L.N1;
    (void)threads_in;
    e0.assign(N1, 0.0);
    if (L.k == 1) {
        // canonical Whitney interpolant: c_e = int_e E0 . t ds (10-point Gauss-Legendre), e0 = M1 c
        std::vector<double> gx, gw;
        gauss_legendre(10, gx, gw);
        std::vector<double> c(N1, 0.0);
        for (int cl = 0; cl < (int)L.c1.size(); ++cl) {
            const Box& b = L.c1[cl].box;
            int d = EDGE_D[L.c1[cl].shape];
            for (int64_t r = 0; r < b.size; ++r) {
                int v[3] = {(int)(r % b.num[0]) + b.lo[0], (int)((r / b.num[0]) % b.num[1]) + b.lo[1],
                            (int)(r / ((int64_t)b.num[0] * b.num[1])) + b.lo[2]};
                double xa[3], dx[3];
                for (int a = 0; a < 3; ++a) {
                    xa[a] = v[a] * L.h;
                    dx[a] = bit(d, a) * L.h;
                }
                double s = 0;
                for (int q = 0; q < 10; ++q) {
                    double u = 0.5 * (gx[q] + 1.0), p[3], E[3];
                    for (int a = 0; a < 3; ++a) p[a] = xa[a] + u * dx[a];
                    E0(p, E, user);
                    s += 0.5 * gw[q] * (E[0] * dx[0] + E[1] * dx[1] + E[2] * dx[2]);
                }
                c[b.offset + r] = s;
            }
        }
        S.M1.matvec(c.data(), e0.data(), 1);
        return 0;
    }
    // k >= 2: L2 load vector with a collapsed (Duffy) Gauss-Legendre rule, 6 points per direction
    std::vector<double> gx6, gw6;
    gauss_legendre(6, gx6, gw6);
    std::vector<F1> F;
    std::vector<bool> ig;
    one_forms(L.k, F, ig);
    const int64_t T = 6LL * L.n * L.n * L.n;
    std::vector<int64_t> g(L.n1);
    RefTet Rs[6];
    for (int s = 0; s < 6; ++s) Rs[s] = ref_tet(s, L.h);
    for (int64_t t = 0; t < T; ++t) {
        int s = (int)(t % 6);
        int64_t cube = t / 6;
        int cc[3] = {(int)(cube % L.n), (int)((cube / L.n) % L.n), (int)(cube / ((int64_t)L.n * L.n))};
        L.tet_dofs1(t, g.data());
        const RefTet& R = Rs[s];
        for (int i1 = 0; i1 < 6; ++i1)
            for (int i2 = 0; i2 < 6; ++i2)
                for (int i3 = 0; i3 < 6; ++i3) {
                    double x1 = 0.5 * (gx6[i1] + 1), x2 = 0.5 * (gx6[i2] + 1), x3 = 0.5 * (gx6[i3] + 1);
                    double wgt = 0.125 * gw6[i1] * gw6[i2] * gw6[i3] * (1 - x1) * (1 - x1) * (1 - x2) * 6.0 * R.vol;
                    double lam[4];
                    lam[1] = x1;
                    lam[2] = (1 - x1) * x2;
                    lam[3] = (1 - x1) * (1 - x2) * x3;
                    lam[0] = 1 - lam[1] - lam[2] - lam[3];
                    double p[3];
                    for (int a = 0; a < 3; ++a) {
                        p[a] = cc[a] * L.h;
                        for (int i = 0; i < 4; ++i) p[a] += lam[i] * R.X[i][a];
                    }
                    double E[3];
                    E0(p, E, user);
                    for (int r = 0; r < L.n1; ++r) {
                        if (g[r] < 0) continue;
                        double v[3];
                        eval1(F[r], lam, R, v);
                        e0[g[r]] += wgt * (v[0] * E[0] + v[1] * E[1] + v[2] * E[2]);
                    }
                }
    }
    return 0;
}

}  // namespace ygm
