// GYM leapfrog step on GB300 (sm_103a): device kernels and the C ABI of include/ygm.h.
//
// One step (state e_n, b_{n-1/2}; Eq. YeeLeapfrog in the GYM form of Eq. preYeeFEECEqns):
//   k_qapply   x = Q1 e_n                                 (shear map Phi^e, Eq. shearMaps)
//   k_curl_b   b_{n+1/2} = b_{n-1/2} - dt C x              (integer curl, Eq. dIsFiniteDiff)
//   k_energy   W_n (every K steps, FP64 compensated)       (telescoping invariant of the leapfrog)
//   k_curlT_e  e_{n+1} = e_n + dt C^T M2 b_{n+1/2}         (shear map Phi^a, Eq. dTIsFiniteDiff)
//   k_source   e_{n+1} -= dt s(t_{n+1/2}) d . Lambda1(x0)  (current term of Eq. allEOM)
// One column (R = 1): k_qapply_s, k_curl_b_s and k_curlT_e_s give one thread to each lattice
// point of a (class, z-plane), with every stencil term a constant 32-bit offset into
// zero-halo padded copies of e, x and b.  R > 1 columns and meshes whose lattice offsets
// overflow 32 bits use k_qapply_p and the range-checked k_curl_b_r / k_curlT_e_r, which give
// each (DoF, column) pair a thread.  Each output element is written by exactly one thread
// in a fixed summation order: results are deterministic, no atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>
#include <string>
#include <vector>

#include "../../include/ygm.h"
#include "builder.h"

namespace {

constexpr int WARPS_PER_BLOCK = 8;
constexpr int BLOCK = 32 * WARPS_PER_BLOCK;

// ------------------------------------------------------------------ device tables
struct DCls {            // a DoF class box (1-form or 2-form)
    int lo[3];
    int num[3];
    long long off;       // global index of the box's first DoF
    long long size;
    long long qoff;      // 1-forms: first packed Q1 value of the class
    int st_begin, st_end;    // 1-forms: stencil slots; 2-forms: curl terms
    int inc_begin, inc_end;  // 1-forms: incident tets
    int pbase;               // 1-forms: first element of the class region in the padded copy of e
    int nup;                 // 1-forms: upper (stored) Q1 slots of the class
};
// Padded copy of e: every 1-form class owns a cube of NP^3 entries indexed by lattice anchor + H
// (anchors -H .. n+H), zero outside the class box, so any Q1 neighbour (|d| <= H per axis) of
// any row is addressed without range checks.
struct PadGeo {
    int H, NP;
};
__device__ __forceinline__ int pad_index(const DCls& C, PadGeo g, int vx, int vy, int vz) {
    return C.pbase + ((vz + g.H) * g.NP + (vy + g.H)) * g.NP + vx + g.H;
}
struct DSlot {           // Q1 stencil slot
    int cls;
    int slot;
    int d[3];
    int upper;
};
struct DTerm {           // one entry of an integer curl row: sign * x[(cls, v + d)]
    int cls;
    int d[3];
    int sign;
};
struct DInc {            // a tet incident to a 1-form entity
    int dcube[3];
    int shape;
    int loc;
};
struct DLoc2 {           // active local 2-form of a tet shape: class and anchor offset
    int cls;
    int off[3];
};
struct DRow {            // one x-row of a class
    int cls;
    int vy, vz;
    int rbase;           // compact index of the row's first element inside the class box
};

struct Tables {
    const DCls* c1;
    const DCls* c2;
    const DSlot* slots;
    const DTerm* terms;
    const DInc* inc;
    const DLoc2* loc2;   // [6][n2a]
    int n;               // cubes per side
    int n1, n2a;
};

__device__ __forceinline__ bool in_box(const DCls& D, int u0, int u1, int u2) {
    return u0 >= 0 && u1 >= 0 && u2 >= 0 && u0 < D.num[0] && u1 < D.num[1] && u2 < D.num[2];
}

// ------------------------------------------------------------------ x = Q1 e, padded e, full rows
// Used with R > 1 columns, and with one column when the upper-triangle lattice of k_qapply_s
// would overflow 32-bit offsets.
// One thread per row.  Q1 is stored by full rows, slot-major per class and z-plane
// (qf[class][slot][z][y][x], zero where the neighbour lies outside its box), and e is read from
// its padded copy, so slot s of every row of a class is the constant offset soff[s] from the
// row's own padded index: the loop body is two loads and one FMA, with no range checks.
constexpr int PBLOCK = 256;
struct PBlk {            // up to PBLOCK consecutive rows of one (class, z-plane)
    int i0;              // first in-plane row index (y * num0 + x) of the block
    int cnt;             // rows in the block
    int num0;            // x extent of the class box
    int pz0;             // padded index of the plane's first anchor (lo_x, lo_y, vz)
    int s_begin, ns;     // slot offsets of the class
    long long q0;        // qf index of the block's first row, slot 0
    long long sstr;      // qf distance between consecutive slots of a row
    long long x0;        // x index of the block's first row
};
// With R = 2^rshift right-hand sides ([N][R] layout) a row owns R consecutive threads, one per
// column; soff is then pre-scaled by R and each Q1 value is shared by the row's R threads.
template <typename real>
__global__ void __launch_bounds__(PBLOCK) k_qapply_p(const PBlk* __restrict__ blks, const int* __restrict__ soff,
                                                     int np, int rshift, const real* __restrict__ qf,
                                                     const real* __restrict__ ep, real* __restrict__ x) {
    extern __shared__ __align__(16) int s_off[];
    const PBlk B = blks[blockIdx.x];
    for (int s = threadIdx.x; s < B.ns; s += blockDim.x) s_off[s] = soff[B.s_begin + s];
    __syncthreads();
    const int row = (int)threadIdx.x >> rshift, col = (int)threadIdx.x & ((1 << rshift) - 1);
    if (row >= B.cnt) return;
    const int i = B.i0 + row;
    const int ry = i / B.num0, rx = i - ry * B.num0;
    const real* __restrict__ e0 = ep + (((long long)(B.pz0 + ry * np + rx) << rshift) + col);
    const real* __restrict__ q = qf + B.q0 + row;
    const long long st = B.sstr;
    real acc = real(0);
    int s = 0;
    // eight slots per round: all sixteen loads are issued before the first FMA needs one
    for (; s + 8 <= B.ns; s += 8) {
        const int4 oa = *reinterpret_cast<const int4*>(&s_off[s]);
        const int4 ob = *reinterpret_cast<const int4*>(&s_off[s + 4]);
        real qv[8], ev[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) qv[u] = __ldg(q + u * st);
        ev[0] = __ldg(e0 + oa.x);
        ev[1] = __ldg(e0 + oa.y);
        ev[2] = __ldg(e0 + oa.z);
        ev[3] = __ldg(e0 + oa.w);
        ev[4] = __ldg(e0 + ob.x);
        ev[5] = __ldg(e0 + ob.y);
        ev[6] = __ldg(e0 + ob.z);
        ev[7] = __ldg(e0 + ob.w);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fma(qv[u], ev[u], acc);
        q += 8 * st;
    }
    for (; s < B.ns; ++s) {
        acc = fma(__ldg(q), __ldg(e0 + s_off[s]), acc);
        q += st;
    }
    x[((B.x0 + row) << rshift) + col] = acc;
}

// ------------------------------------------------------------------ x = Q1 e, upper triangle, plane sweep
// Q1 stored once per symmetric pair: row (c, v) keeps its upper slots (neighbours at or after
// itself in (dz, dy, dx, class) order) in qs[c][slot][vz][vy][vx] on the common anchor lattice;
// its lower slots are the neighbours' upper slots, i.e. the same array at a constant offset
// from the row.  Every slot is therefore one 32-bit element offset for Q1 and one for the padded
// e, and the loop body is two loads and one FMA.  Lower slots point to rows at dz <= 0, and the
// blocks are ordered by z-plane, so those values were streamed from HBM by the blocks of the
// same or the previous planes shortly before and can be read again from L2: the upper loads
// carry an L2 evict-last hint (the value has one more reader), the lower loads evict-first
// (last reader).  Lattice points outside the row's box (PEC-removed rows, and the wrap-around of
// neighbour offsets) hold finite values that multiply a zero of the padded e.
// Slot order per class: the upper slots, then the lower ones, each group in padded-e order so
// consecutive loads of e share L1 lines.
// FP32 sums are compensated (Kahan): the stencil sum cancels strongly (the rows of an
// approximate inverse of an ill-conditioned mass matrix), and the plain FP32 sum is the largest
// rounding term of the FP32 step.  The extra adds are hidden behind the memory stream.
// ENERGY: every row also adds e_i x_i to a per-block FP64 partial (the e^T Q1 e half of W_n).
constexpr int SBLOCK = 256;
struct SBlk {            // up to SBLOCK consecutive lattice points (vy * NX + vx) of one (class, z-plane)
    long long q0;        // qs index of the plane's first lattice point (class base + vz * NY * NX)
    int cls;
    int vz;
    int t0;              // first lattice point of the block inside the plane
    int cnt;
};
struct SymGeo {
    int NX;              // lattice row length (multiple of 8)
    int H, NP;           // padded e geometry
};
template <typename real>
__device__ __forceinline__ real ld_l2hint(const real* p, unsigned long long pol) {
    real v;
    if constexpr (std::is_same<real, float>::value)
        asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    else
        asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
// running sum: compensated for float, plain FMA for double
template <typename real>
struct KSum {
    real s = real(0), c = real(0);
    __device__ __forceinline__ void add(real q, real e) {
        if constexpr (std::is_same<real, float>::value) {
            const real y = fma(q, e, -c);
            const real t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s = fma(q, e, s);
        }
    }
};
// sixteen slots per round: all 32 loads are in flight before the first of them is consumed (the
// kernel is bound by load latency; measured 212 us against 233 us with eight at N=32, k=2)
template <typename real>
__device__ __forceinline__ void qs_run(KSum<real>& a, const int2* s_o2, int s, int send, const real* q, const real* e0,
                                       unsigned long long pol) {
    constexpr int U = 16;
    for (; s + U <= send; s += U) {
        real qv[U], ev[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int2 o = s_o2[s + u];
            qv[u] = ld_l2hint(q + o.x, pol);
            ev[u] = __ldg(e0 + o.y);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) a.add(qv[u], ev[u]);
    }
    for (; s < send; ++s) {
        const int2 o = s_o2[s];
        a.add(ld_l2hint(q + o.x, pol), __ldg(e0 + o.y));
    }
}

// ------------------------------------------------------------------ curls on the padded lattice, one column
// Same blocks as k_qapply_s (SBLOCK lattice points of one class and z-plane).  x and b keep
// zero-halo padded copies in the geometry of the padded e, so every curl term is a constant
// 32-bit offset from the row's padded index and the loops carry no range checks.  The terms
// are summed in the order of the range-checked kernels, so both give identical results.
struct CTermL {          // one entry of an integer curl row: sign * xp[row + off]
    int off;
    int sign;
};
template <typename real>
struct WTermL {          // one merged C^T M2 weight: w * bp[row + off]
    int off;
    real w;
};
__device__ __forceinline__ int pad_row(PadGeo g, int vx, int vy, int vz) {
    return ((vz + g.H) * g.NP + (vy + g.H)) * g.NP + vx + g.H;
}
// A step size in two parts, hi + lo = ctau to ~2^-48 relative: hi is the nearest value of the
// state type, lo the rest (0 in FP64).  An FP32 update with hi alone would run the leapfrog at a
// step rounded by up to 6e-8, a systematic phase drift that grows with the number of steps.
template <typename real>
struct Tau {
    real hi, lo;
};
template <typename real>
static Tau<real> split_tau(double t) {
    const real hi = (real)t;
    return Tau<real>{hi, (real)(t - (double)hi)};
}
// b_out = b_in - ctau C x; also bp <- b_out (the rows of one block)
template <typename real>
__device__ __forceinline__ void curl_b_rows(const SBlk& B, const DCls* __restrict__ c2, const CTermL* __restrict__ terms,
                                            PadGeo g, int NX, const real* __restrict__ xp, const real* b_in, real* b_out,
                                            real* __restrict__ bp, Tau<real> ctau) {
    const DCls C = c2[B.cls];
    if ((int)threadIdx.x >= B.cnt) return;
    const int t = B.t0 + (int)threadIdx.x;
    const int vy = t / NX, vx = t - vy * NX;
    const int rx = vx - C.lo[0], ry = vy - C.lo[1];
    if ((unsigned)rx >= (unsigned)C.num[0] || (unsigned)ry >= (unsigned)C.num[1]) return;
    const int p = pad_row(g, vx, vy, B.vz);
    const long long gi = C.off + ((long long)(B.vz - C.lo[2]) * C.num[1] + ry) * C.num[0] + rx;
    const real bo = b_in[gi];
    // at most three terms (Whitney incidence) or one (curl of a higher-order 1-form): every load is
    // issued before the first sum, which keeps the term order
    const int nt = C.st_end - C.st_begin;
    real xv[3];
    int sg[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        xv[u] = real(0);
        sg[u] = 0;
        if (u < nt) {
            const CTermL T = terms[C.st_begin + u];
            xv[u] = __ldg(xp + p + T.off);
            sg[u] = T.sign;
        }
    }
    real acc = real(0);
#pragma unroll
    for (int u = 0; u < 3; ++u)
        if (u < nt) acc += sg[u] > 0 ? xv[u] : -xv[u];
    const real v = fma(-ctau.lo, acc, fma(-ctau.hi, acc, bo));
    b_out[gi] = v;
    bp[C.pbase + p] = v;
}
// Programmatic dependent launch between the kernels of a one-column step (k_qapply_s ->
// k_curl_b_s -> k_curlT_e_s -> k_qapply_s ...).  Each of them lets the next grid launch once its
// own blocks are all running (pdl_trigger) and, after loading only constant tables, waits for the
// previous grid to complete with its writes visible (pdl_wait) before it reads the previous
// kernel's output or writes anything.  So no kernel touches mutable data before its predecessor
// has finished, and each predecessor had itself waited for its own.  Under an ordinary launch both
// instructions do nothing.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename real>
__global__ void __launch_bounds__(SBLOCK) k_curl_b_s(const SBlk* __restrict__ blks, const DCls* __restrict__ c2,
                                                     const CTermL* __restrict__ terms, PadGeo g, int NX,
                                                     const real* __restrict__ xp, const real* b_in, real* b_out,
                                                     real* __restrict__ bp, Tau<real> ctau) {
    pdl_trigger();
    pdl_wait();
    curl_b_rows(blks[blockIdx.x], c2, terms, g, NX, xp, b_in, b_out, bp, ctau);
}
// A dipole source DoF inside a block of k_curlT_e_s: thread, source index, weight d . Lambda1_i(x0).
template <typename real>
struct SrcE {
    int tid;
    int src;
    real w;
};
// e += ctau C^T M2 b (uniform mu), from the padded b; also ep <- e.  With amp != NULL the dipole
// currents of this step are subtracted in the same pass: e_i -= amp[s] w_i for the entries
// sbeg[block] .. sbeg[block + 1] (amp[s] = dt s_s(t_{n+1/2}), host FP64).  Blocks of classes that
// carry no curl appear in the launch only when a source DoF lies in them; their stencil is empty.
// the rows of one block; s_t holds the class's merged terms (loaded by the caller), item is the
// block's index in the source tables
template <typename real>
__device__ __forceinline__ void curlT_e_rows(const SBlk& B, const DCls* __restrict__ c1, const WTermL<real>* s_t, int nt,
                                             PadGeo g, int NX, const real* __restrict__ bp, real* __restrict__ e,
                                             Tau<real> ctau, real* __restrict__ ep, const int* __restrict__ sbeg,
                                             const SrcE<real>* __restrict__ sent, const double* __restrict__ amp, int item) {
    const DCls C = c1[B.cls];
    if ((int)threadIdx.x >= B.cnt) return;
    const int t = B.t0 + (int)threadIdx.x;
    const int vy = t / NX, vx = t - vy * NX;
    const int rx = vx - C.lo[0], ry = vy - C.lo[1];
    if ((unsigned)rx >= (unsigned)C.num[0] || (unsigned)ry >= (unsigned)C.num[1]) return;
    const int p = pad_row(g, vx, vy, B.vz);
    const real* __restrict__ b0 = bp + p;
    real acc = real(0);
    int s = 0;
    for (; s + 8 <= nt; s += 8) {
        real bv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) bv[u] = __ldg(b0 + s_t[s + u].off);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fma(s_t[s + u].w, bv[u], acc);
    }
    for (; s < nt; ++s) acc = fma(s_t[s].w, __ldg(b0 + s_t[s].off), acc);
    const long long gi = C.off + ((long long)(B.vz - C.lo[2]) * C.num[1] + ry) * C.num[0] + rx;
    real v = fma(ctau.lo, acc, fma(ctau.hi, acc, e[gi]));
    if (amp)
        for (int i = sbeg[item]; i < sbeg[item + 1]; ++i)
            if (sent[i].tid == (int)threadIdx.x) v -= (real)amp[sent[i].src] * sent[i].w;
    e[gi] = v;
    ep[C.pbase + p] = v;
}
template <typename real>
__global__ void __launch_bounds__(SBLOCK) k_curlT_e_s(const SBlk* __restrict__ blks, const DCls* __restrict__ c1,
                                                      const int* __restrict__ pbeg, const WTermL<real>* __restrict__ terms,
                                                      PadGeo g, int NX, const real* __restrict__ bp, real* __restrict__ e,
                                                      Tau<real> ctau, real* __restrict__ ep, const int* __restrict__ sbeg,
                                                      const SrcE<real>* __restrict__ sent, const double* __restrict__ amp) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    WTermL<real>* s_t = reinterpret_cast<WTermL<real>*>(s_raw);
    const SBlk B = blks[blockIdx.x];
    const int tb = pbeg[B.cls], nt = pbeg[B.cls + 1] - tb;
    for (int s = threadIdx.x; s < nt; s += blockDim.x) s_t[s] = terms[tb + s];
    __syncthreads();
    pdl_trigger();
    pdl_wait();
    curlT_e_rows(B, c1, s_t, nt, g, NX, bp, e, ctau, ep, sbeg, sent, amp, (int)blockIdx.x);
}

// ep (padded) <- e (compact), one block per (class, z-plane)
template <typename real>
__global__ void k_pad_e(const DCls* __restrict__ c1, const int2* __restrict__ planes, PadGeo g, int rshift,
                        const real* __restrict__ e, real* __restrict__ ep) {
    const int2 P = planes[blockIdx.x];     // (class, vz)
    const DCls C = c1[P.x];
    const int plane = C.num[0] * C.num[1];
    const long long base = C.off + (long long)(P.y - C.lo[2]) * plane;
    const int R = 1 << rshift;
    for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < plane * R; t += gridDim.y * blockDim.x) {
        const int i = t >> rshift, col = t & (R - 1);
        const int ry = i / C.num[0], rx = i - ry * C.num[0];
        ep[((long long)pad_index(C, g, C.lo[0] + rx, C.lo[1] + ry, P.y) << rshift) + col] = e[((base + i) << rshift) + col];
    }
}

// ------------------------------------------------------------------ x = Q1 e, symmetric storage
constexpr int TY = 4;
struct QSlot {
    int ux0, uy0, uz0;   // slot offset minus the neighbour box origin
    int nx, ny, nz;      // neighbour box
    long long ebase;     // first e index of the neighbour class
    long long qbase;     // upper: own qoff + slot * own size; lower: neighbour qoff + slot * its size
    int upper;
    int pad;
};
// ------------------------------------------------------------------ x = Q1 e, block per (z, class)
// A block owns one z-plane of one class; its warps take y-tiles of TY rows (32 lanes along x).
// The class's slot descriptors are staged in shared memory once; the slot loop is straight
// line (validity folded into predicates) and unrolled, so many independent loads are in
// flight per thread -- the kernel is meant to stream Q1 at HBM speed.
struct QBlock {
    int cls;
    int vz;
};
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_qapply_b(const DCls* __restrict__ c1, const QSlot* __restrict__ slots,
                                                    const QBlock* __restrict__ blocks, int max_slots,
                                                    const real* __restrict__ q, const real* __restrict__ e,
                                                    real* __restrict__ x) {
    extern __shared__ long long smem_q[];
    long long (*s_l)[2] = reinterpret_cast<long long (*)[2]>(smem_q);            // ebase, qbase
    int (*s_i)[8] = reinterpret_cast<int (*)[8]>(smem_q + 2 * (size_t)max_slots); // ux0 uy0 uz0 nx ny nz upper -
    const QBlock Bk = blocks[blockIdx.x];
    const DCls C = c1[Bk.cls];
    const int ns = C.st_end - C.st_begin;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const QSlot S = slots[C.st_begin + s];
        s_i[s][0] = S.ux0;
        s_i[s][1] = S.uy0;
        s_i[s][2] = S.uz0;
        s_i[s][3] = S.nx;
        s_i[s][4] = S.ny;
        s_i[s][5] = S.nz;
        s_i[s][6] = S.upper;
        s_i[s][7] = 0;
        s_l[s][0] = S.ebase;
        s_l[s][1] = S.qbase;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int rz = Bk.vz - C.lo[2];
    const int cnx = C.num[0];
    for (int ry0 = warp * TY; ry0 < C.num[1]; ry0 += nwarps * TY) {
        const int vy0 = C.lo[1] + ry0;
        const int nrows = min(TY, C.num[1] - ry0);
        for (int x0 = 0; x0 < cnx; x0 += 32) {
            const int ix = x0 + lane;
            const bool act = ix < cnx;
            const int vx = C.lo[0] + ix;
            const long long own0 = ((long long)rz * C.num[1] + ry0) * cnx + ix;   // own index, row t = 0
            real acc[TY];
#pragma unroll
            for (int t = 0; t < TY; ++t) acc[t] = real(0);
#pragma unroll 4
            for (int s = 0; s < ns; ++s) {
                const int4 a0 = *reinterpret_cast<const int4*>(&s_i[s][0]);     // ux0 uy0 uz0 nx
                const int4 a1 = *reinterpret_cast<const int4*>(&s_i[s][4]);     // ny nz upper -
                const longlong2 bb = *reinterpret_cast<const longlong2*>(&s_l[s][0]);
                const int uz = Bk.vz + a0.z;
                const int uy0 = vy0 + a0.y;
                const int tlo = -uy0, thi = min(nrows, a1.x - uy0);           // valid rows: tlo <= t < thi
                const int ux = vx + a0.x;
                const bool okl = act && (unsigned)ux < (unsigned)a0.w && (unsigned)uz < (unsigned)a1.y;
                const long long nb0 = ((long long)uz * a1.x + uy0) * a0.w + ux;
                const long long qi0 = a1.z ? bb.y + own0 : bb.y + nb0;
                const long long qst = a1.z ? cnx : a0.w;
                const long long ei0 = bb.x + nb0;
#pragma unroll
                for (int t = 0; t < TY; ++t) {
                    const bool ok = okl && t >= tlo && t < thi;
                    const real qv = ok ? __ldg(q + qi0 + t * qst) : real(0);
                    const real ev = ok ? __ldg(e + ei0 + (long long)t * a0.w) : real(0);
                    acc[t] = fma(qv, ev, acc[t]);
                }
            }
            if (act) {
#pragma unroll
                for (int t = 0; t < TY; ++t)
                    if (t < nrows) x[C.off + own0 + (long long)t * cnx] = acc[t];
            }
        }
    }
}

// ------------------------------------------------------------------ e += ctau C^T M2 b, merged stencil
// With a uniform permeability, C^T M2 is a constant-coefficient stencil from the curl-carrying
// 2-forms to each 1-form class: the contributions of all tets around the entity are summed on
// the host into one weight per (2-form class, offset).
template <typename real>
struct PTerm {
    int ux0, uy0, uz0;
    int nx, ny, nz;
    long long bbase;
    real w;
};
// ------------------------------------------------------------------ e += ctau C^T M2 b
// Per tet T containing the entity: (1/mu_T) sum_r W[loc][r] b_T[r], W = C_loc^T M2_loc on the
// curl-carrying local 2-forms (the divergence part of b never changes: C has no row there).
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_curlT_e(Tables tb, const DRow* __restrict__ rows, int nrows,
                                                   const real* __restrict__ W, const real* __restrict__ b,
                                                   const real* __restrict__ inv_mu, real* e, real ctau, real* ep,
                                                   PadGeo g) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * WARPS_PER_BLOCK + warp;
    if (row >= nrows) return;
    const DRow R = rows[row];
    const DCls C = tb.c1[R.cls];
    const int n = tb.n, n2a = tb.n2a;
    for (int x0 = 0; x0 < C.num[0]; x0 += 32) {
        const int ix = x0 + lane;
        if (ix >= C.num[0]) break;
        const int vx = C.lo[0] + ix;
        real acc = real(0);
        for (int ic = C.inc_begin; ic < C.inc_end; ++ic) {
            const DInc I = tb.inc[ic];
            const int cx = vx + I.dcube[0], cy = R.vy + I.dcube[1], cz = R.vz + I.dcube[2];
            const real* Wr = W + (long long)I.loc * n2a;
            const DLoc2* L2 = tb.loc2 + I.shape * n2a;
            real t = real(0);
            for (int r = 0; r < n2a; ++r) {
                const DLoc2 Lr = L2[r];
                const DCls D = tb.c2[Lr.cls];
                const int ux = cx + Lr.off[0] - D.lo[0], uy = cy + Lr.off[1] - D.lo[1], uz = cz + Lr.off[2] - D.lo[2];
                if (!in_box(D, ux, uy, uz)) continue;    // PEC: boundary faces carry no DoF
                t = fma(__ldg(Wr + r), __ldg(b + D.off + ((long long)uz * D.num[1] + uy) * D.num[0] + ux), t);
            }
            if (inv_mu) t *= __ldg(inv_mu + 6 * ((long long)cx + (long long)n * (cy + (long long)n * cz)) + I.shape);
            acc += t;
        }
        const long long gi = C.off + R.rbase + ix;
        const real v = e[gi] + ctau * acc;
        e[gi] = v;
        if (ep) ep[pad_index(C, g, vx, R.vy, R.vz)] = v;
    }
}

// ------------------------------------------------------------------ e += ctau C^T M2 b, block per (z, class)
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_curlT_e_b(const DCls* __restrict__ c1, const int* __restrict__ pbeg,
                                                     const PTerm<real>* __restrict__ terms, const QBlock* __restrict__ blocks,
                                                     int max_terms, const real* __restrict__ b, real* e, real ctau,
                                                     real* ep, PadGeo g) {
    extern __shared__ long long smem_p[];
    long long* s_b = smem_p;                                               // bbase
    real* s_w = reinterpret_cast<real*>(smem_p + max_terms);                // weight
    int (*s_i)[6] = reinterpret_cast<int (*)[6]>(s_w + max_terms + (max_terms & 1));
    const QBlock Bk = blocks[blockIdx.x];
    const DCls C = c1[Bk.cls];
    const int tb = pbeg[Bk.cls], nt = pbeg[Bk.cls + 1] - tb;
    for (int s = threadIdx.x; s < nt; s += blockDim.x) {
        const PTerm<real> P = terms[tb + s];
        s_b[s] = P.bbase;
        s_w[s] = P.w;
        s_i[s][0] = P.ux0;
        s_i[s][1] = P.uy0;
        s_i[s][2] = P.uz0;
        s_i[s][3] = P.nx;
        s_i[s][4] = P.ny;
        s_i[s][5] = P.nz;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rz = Bk.vz - C.lo[2];
    for (int ry0 = warp * TY; ry0 < C.num[1]; ry0 += WARPS_PER_BLOCK * TY) {
        const int vy0 = C.lo[1] + ry0;
        const int nrows = min(TY, C.num[1] - ry0);
        for (int x0 = 0; x0 < C.num[0]; x0 += 32) {
            const int ix = x0 + lane;
            const bool act = ix < C.num[0];
            const int vx = C.lo[0] + ix;
            real acc[TY];
#pragma unroll
            for (int t = 0; t < TY; ++t) acc[t] = real(0);
#pragma unroll 4
            for (int s = 0; s < nt; ++s) {
                const int ux = vx + s_i[s][0];
                const int uz = Bk.vz + s_i[s][2];
                const int nx = s_i[s][3], ny = s_i[s][4];
                const bool okxz = act && (unsigned)ux < (unsigned)nx && (unsigned)uz < (unsigned)s_i[s][5];
                const long long nb0 = s_b[s] + ((long long)uz * ny + vy0 + s_i[s][1]) * nx + ux;
                const real w = s_w[s];
#pragma unroll
                for (int t = 0; t < TY; ++t) {
                    const int uy = vy0 + t + s_i[s][1];
                    const bool ok = okxz && t < nrows && (unsigned)uy < (unsigned)ny;
                    const real bv = ok ? __ldg(b + nb0 + (long long)t * nx) : real(0);
                    acc[t] = fma(w, bv, acc[t]);
                }
            }
            if (act) {
                const long long g0 = C.off + ((long long)rz * C.num[1] + ry0) * C.num[0] + ix;
#pragma unroll
                for (int t = 0; t < TY; ++t)
                    if (t < nrows) {
                        const long long gi = g0 + (long long)t * C.num[0];
                        const real v = e[gi] + ctau * acc[t];
                        e[gi] = v;
                        if (ep) ep[pad_index(C, g, vx, vy0 + t, Bk.vz)] = v;
                    }
            }
        }
    }
}

// ------------------------------------------------------------------ b_out = b_in - ctau C x, block per (z, class)
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_curl_b_b(const DCls* __restrict__ c1, const DCls* __restrict__ c2,
                                                    const DTerm* __restrict__ terms, const QBlock* __restrict__ blocks,
                                                    const real* __restrict__ x, const real* b_in, real* b_out, real ctau) {
    const QBlock Bk = blocks[blockIdx.x];
    const DCls C = c2[Bk.cls];
    const int nt = C.st_end - C.st_begin;
    // at most three signed terms per row (Whitney incidence) or one (curl of a higher-order 1-form)
    int t_ux0[3], t_uy0[3], t_uz0[3], t_nx[3], t_ny[3], t_nz[3], t_sg[3];
    long long t_off[3];
    for (int s = 0; s < 3; ++s) {
        if (s < nt) {
            const DTerm Tm = terms[C.st_begin + s];
            const DCls D = c1[Tm.cls];
            t_ux0[s] = Tm.d[0] - D.lo[0];
            t_uy0[s] = Tm.d[1] - D.lo[1];
            t_uz0[s] = Tm.d[2] - D.lo[2];
            t_nx[s] = D.num[0];
            t_ny[s] = D.num[1];
            t_nz[s] = D.num[2];
            t_off[s] = D.off;
            t_sg[s] = Tm.sign;
        } else {
            t_ux0[s] = t_uy0[s] = t_uz0[s] = 0;
            t_nx[s] = t_ny[s] = t_nz[s] = 0;      // never valid
            t_off[s] = 0;
            t_sg[s] = 0;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rz = Bk.vz - C.lo[2];
    for (int ry = warp; ry < C.num[1]; ry += WARPS_PER_BLOCK) {
        const int vy = C.lo[1] + ry;
        for (int x0 = 0; x0 < C.num[0]; x0 += 32) {
            const int ix = x0 + lane;
            if (ix >= C.num[0]) break;
            const int vx = C.lo[0] + ix;
            real acc = real(0);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int ux = vx + t_ux0[s], uy = vy + t_uy0[s], uz = Bk.vz + t_uz0[s];
                const bool ok = (unsigned)ux < (unsigned)t_nx[s] && (unsigned)uy < (unsigned)t_ny[s] &&
                                (unsigned)uz < (unsigned)t_nz[s];
                const real xv = ok ? __ldg(x + t_off[s] + ((long long)uz * t_ny[s] + uy) * t_nx[s] + ux) : real(0);
                acc += t_sg[s] > 0 ? xv : -xv;
            }
            const long long g = C.off + ((long long)rz * C.num[1] + ry) * C.num[0] + ix;
            b_out[g] = b_in[g] - ctau * acc;
        }
    }
}

// ------------------------------------------------------------------ point-dipole sources
// amp[s] = dt * s_s(t_{n+1/2}) is computed on the host in FP64 for every step of a call.
struct DSrc {
    int begin, end;      // into the (dof, weight) lists
};
template <typename real>
__global__ void k_source(const DSrc* __restrict__ src, int nsrc, const long long* __restrict__ dofs,
                         const int* __restrict__ pdofs, const real* __restrict__ w, const double* __restrict__ amp,
                         real* e, real* ep) {
    for (int s = 0; s < nsrc; ++s) {
        const DSrc S = src[s];
        const real a = (real)amp[s];
        for (int i = S.begin + threadIdx.x; i < S.end; i += blockDim.x) {
            const real v = e[dofs[i]] - a * w[i];
            e[dofs[i]] = v;
            ep[pdofs[i]] = v;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ R > 1 right-hand sides
// State vectors are [N][R] (R = 2^rshift contiguous columns).  These kernels give every
// (DoF, column) pair its own thread inside a block that owns one (class, z-plane): consecutive
// threads run over the R columns of one DoF, so every gather of a neighbour reads R contiguous
// values.  The operator tables are the ones of the single-column kernels.

// b_out = b_in - ctau C x
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_curl_b_r(const DCls* __restrict__ c1, const DCls* __restrict__ c2,
                                                    const DTerm* __restrict__ terms, const QBlock* __restrict__ blocks,
                                                    int rshift, const real* __restrict__ x, const real* b_in,
                                                    real* b_out, real ctau) {
    const QBlock Bk = blocks[blockIdx.x];
    const DCls C = c2[Bk.cls];
    const int nt = C.st_end - C.st_begin;
    int t_ux0[3], t_uy0[3], t_uz0[3], t_nx[3], t_ny[3], t_nz[3], t_sg[3];
    long long t_off[3];
    for (int s = 0; s < 3; ++s) {
        if (s < nt) {
            const DTerm Tm = terms[C.st_begin + s];
            const DCls D = c1[Tm.cls];
            t_ux0[s] = Tm.d[0] - D.lo[0];
            t_uy0[s] = Tm.d[1] - D.lo[1];
            t_uz0[s] = Tm.d[2] - D.lo[2];
            t_nx[s] = D.num[0];
            t_ny[s] = D.num[1];
            t_nz[s] = D.num[2];
            t_off[s] = D.off;
            t_sg[s] = Tm.sign;
        } else {
            t_ux0[s] = t_uy0[s] = t_uz0[s] = 0;
            t_nx[s] = t_ny[s] = t_nz[s] = 0;      // never valid
            t_off[s] = 0;
            t_sg[s] = 0;
        }
    }
    const int plane = C.num[0] * C.num[1], R = 1 << rshift;
    const long long base = C.off + (long long)(Bk.vz - C.lo[2]) * plane;
    for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < plane * R; t += gridDim.y * blockDim.x) {
        const int i = t >> rshift, col = t & (R - 1);
        const int ry = i / C.num[0], rx = i - ry * C.num[0];
        const int vx = C.lo[0] + rx, vy = C.lo[1] + ry;
        real acc = real(0);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int ux = vx + t_ux0[s], uy = vy + t_uy0[s], uz = Bk.vz + t_uz0[s];
            const bool ok = (unsigned)ux < (unsigned)t_nx[s] && (unsigned)uy < (unsigned)t_ny[s] &&
                            (unsigned)uz < (unsigned)t_nz[s];
            const real xv =
                ok ? __ldg(x + ((t_off[s] + ((long long)uz * t_ny[s] + uy) * t_nx[s] + ux) << rshift) + col) : real(0);
            acc += t_sg[s] > 0 ? xv : -xv;
        }
        const long long g = ((base + i) << rshift) + col;
        b_out[g] = b_in[g] - ctau * acc;
    }
}

// e += ctau C^T M2 b with the merged constant stencil (uniform mu); writes the padded copy too
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_curlT_e_r(const DCls* __restrict__ c1, const int* __restrict__ pbeg,
                                                     const PTerm<real>* __restrict__ terms, const QBlock* __restrict__ blocks,
                                                     int rshift, const real* __restrict__ b, real* e, real ctau, real* ep,
                                                     PadGeo g) {
    extern __shared__ long long smem_r[];
    const QBlock Bk = blocks[blockIdx.x];
    const DCls C = c1[Bk.cls];
    const int tb = pbeg[Bk.cls], nt = pbeg[Bk.cls + 1] - tb;
    PTerm<real>* s_t = reinterpret_cast<PTerm<real>*>(smem_r);
    for (int s = threadIdx.x; s < nt; s += blockDim.x) s_t[s] = terms[tb + s];
    __syncthreads();
    const int plane = C.num[0] * C.num[1], R = 1 << rshift;
    const long long base = C.off + (long long)(Bk.vz - C.lo[2]) * plane;
    for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < plane * R; t += gridDim.y * blockDim.x) {
        const int i = t >> rshift, col = t & (R - 1);
        const int ry = i / C.num[0], rx = i - ry * C.num[0];
        const int vx = C.lo[0] + rx, vy = C.lo[1] + ry;
        real acc = real(0);
        // eight terms per round, loads first (an out-of-range term adds w * 0 = 0 exactly)
        for (int s0 = 0; s0 < nt; s0 += 8) {
            real bv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                bv[u] = real(0);
                if (s0 + u < nt) {
                    const PTerm<real>& P = s_t[s0 + u];
                    const int ux = vx + P.ux0, uy = vy + P.uy0, uz = Bk.vz + P.uz0;
                    if ((unsigned)ux < (unsigned)P.nx && (unsigned)uy < (unsigned)P.ny && (unsigned)uz < (unsigned)P.nz)
                        bv[u] = __ldg(b + ((P.bbase + ((long long)uz * P.ny + uy) * P.nx + ux) << rshift) + col);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (s0 + u < nt) acc = fma(s_t[s0 + u].w, bv[u], acc);
        }
        const long long gi = ((base + i) << rshift) + col;
        const real v = e[gi] + ctau * acc;
        e[gi] = v;
        if (ep) ep[((long long)pad_index(C, g, vx, vy, Bk.vz) << rshift) + col] = v;
    }
}

// e += ctau C^T M2 b tet by tet (per-tet 1/mu); writes the padded copy too
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_curlT_e_rt(Tables tb, const QBlock* __restrict__ blocks, int rshift,
                                                      const real* __restrict__ W, const real* __restrict__ b,
                                                      const real* __restrict__ inv_mu, real* e, real ctau, real* ep,
                                                      PadGeo g) {
    const QBlock Bk = blocks[blockIdx.x];
    const DCls C = tb.c1[Bk.cls];
    const int n = tb.n, n2a = tb.n2a;
    const int plane = C.num[0] * C.num[1], R = 1 << rshift;
    const long long base = C.off + (long long)(Bk.vz - C.lo[2]) * plane;
    for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < plane * R; t += gridDim.y * blockDim.x) {
        const int i = t >> rshift, col = t & (R - 1);
        const int ry = i / C.num[0], rx = i - ry * C.num[0];
        const int vx = C.lo[0] + rx, vy = C.lo[1] + ry;
        real acc = real(0);
        for (int ic = C.inc_begin; ic < C.inc_end; ++ic) {
            const DInc I = tb.inc[ic];
            const int cx = vx + I.dcube[0], cy = vy + I.dcube[1], cz = Bk.vz + I.dcube[2];
            const real* Wr = W + (long long)I.loc * n2a;
            const DLoc2* L2 = tb.loc2 + I.shape * n2a;
            real tq = real(0);
            for (int r = 0; r < n2a; ++r) {
                const DLoc2 Lr = L2[r];
                const DCls D = tb.c2[Lr.cls];
                const int ux = cx + Lr.off[0] - D.lo[0], uy = cy + Lr.off[1] - D.lo[1], uz = cz + Lr.off[2] - D.lo[2];
                if (!in_box(D, ux, uy, uz)) continue;    // PEC: boundary faces carry no DoF
                tq = fma(__ldg(Wr + r), __ldg(b + ((D.off + ((long long)uz * D.num[1] + uy) * D.num[0] + ux) << rshift) + col), tq);
            }
            if (inv_mu) tq *= __ldg(inv_mu + 6 * ((long long)cx + (long long)n * (cy + (long long)n * cz)) + I.shape);
            acc += tq;
        }
        const long long gi = ((base + i) << rshift) + col;
        const real v = e[gi] + ctau * acc;
        e[gi] = v;
        if (ep) ep[((long long)pad_index(C, g, vx, vy, Bk.vz) << rshift) + col] = v;
    }
}

// ------------------------------------------------------------------ FP64 compensated reductions
struct Neu {
    double s, c;
};
__device__ __forceinline__ Neu neu_add(Neu a, double v) {
    double t = a.s + v;
    if (fabs(a.s) >= fabs(v))
        a.c += (a.s - t) + v;
    else
        a.c += (v - t) + a.s;
    a.s = t;
    return a;
}
__device__ __forceinline__ Neu neu_merge(Neu a, Neu b) {
    Neu r = neu_add(a, b.s);
    r.c += b.c;
    return r;
}
__device__ Neu block_reduce(Neu v) {
    __shared__ double ss[32], sc[32];
    for (int o = 16; o > 0; o >>= 1) {
        Neu u{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
        v = neu_merge(v, u);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        ss[warp] = v.s;
        sc[warp] = v.c;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? Neu{ss[lane], sc[lane]} : Neu{0.0, 0.0};
        for (int o = 16; o > 0; o >>= 1) {
            Neu u{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
            v = neu_merge(v, u);
        }
    }
    return v;
}

// x = Q1 e on the upper-triangle lattice (see the storage notes above k_qapply_s's helpers)
template <typename real, bool ENERGY>
__global__ void __launch_bounds__(SBLOCK, 1) k_qapply_s(const SBlk* __restrict__ blks, const DCls* __restrict__ c1,
                                                     const int2* __restrict__ soff2, SymGeo g,
                                                     const real* __restrict__ qs, const real* __restrict__ ep,
                                                     real* __restrict__ x, real* __restrict__ xp, double2* part) {
    extern __shared__ __align__(16) int2 s_o2[];
    const SBlk B = blks[blockIdx.x];
    const DCls C = c1[B.cls];
    const int ns = C.st_end - C.st_begin;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) s_o2[s] = soff2[C.st_begin + s];
    __syncthreads();
    pdl_trigger();
    pdl_wait();
    const int t = B.t0 + (int)threadIdx.x;
    const int vy = t / g.NX, vx = t - vy * g.NX;
    const int rx = vx - C.lo[0], ry = vy - C.lo[1];
    const bool row = (int)threadIdx.x < B.cnt && (unsigned)rx < (unsigned)C.num[0] && (unsigned)ry < (unsigned)C.num[1];
    if (!ENERGY && !row) return;
    Neu w{0.0, 0.0};
    if (row) {
        unsigned long long keep, drop;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(drop));
        const real* __restrict__ q = qs + (B.q0 + t);
        const int pe = C.pbase + ((B.vz + g.H) * g.NP + (vy + g.H)) * g.NP + vx + g.H;
        const real* __restrict__ e0 = ep + pe;
        KSum<real> a;
        qs_run(a, s_o2, 0, C.nup, q, e0, keep);
        qs_run(a, s_o2, C.nup, ns, q, e0, drop);
        x[C.off + ((long long)(B.vz - C.lo[2]) * C.num[1] + ry) * C.num[0] + rx] = a.s;
        xp[pe] = a.s;
        if (ENERGY) w = neu_add(w, (double)e0[0] * (double)a.s);
    }
    if (ENERGY) {
        w = block_reduce(w);
        if (threadIdx.x == 0) part[blockIdx.x] = make_double2(w.s, w.c);
    }
}

// x = Q1 e on the upper-triangle lattice with the Q1 stream moved off the threads' load path.
// A block's slot s reads the SBLOCK consecutive lattice entries qs[q0 + t0 + o.x(s) + 0 .. SBLOCK-1],
// one contiguous run per slot.  A producer warp copies the runs into a ring of nst shared-memory
// stages (cp.async.bulk, QtCfg::SPS slots per stage, one lane per slot; completion counted in bytes on
// the stage's "full" mbarrier) while SBLOCK consumer threads, one per row as in k_qapply_s, read
// their Q1 values from shared memory and gather e; each consumer warp signals a consumed stage on
// its "empty" mbarrier, which the producer waits for before refilling it.  The warps never wait
// for each other otherwise.  The sum runs over the same slots in the same order as k_qapply_s,
// so both give bit-identical x.  A lower slot's run starts wherever its neighbour offset puts it:
// the copy starts at the 16-byte boundary below and takes 16 bytes more, and the thread indexes
// from the remainder.  Upper runs carry the L2 evict-last hint, lower runs evict-first, as in
// k_qapply_s.  Every wait has an iteration cap: a warp that gives up sets bit QT_ERR_BIT of *err
// and stops; the producer then waits (capped) for the copies it still has in flight, so that no
// copy lands after the block has gone.  The qs guard band keeps every run, with its extra 16
// bytes, inside the array.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <typename real>
struct QtCfg {
    static constexpr int SPS = 64 / (int)sizeof(real);             // slots per stage: 16 (FP32), 8 (FP64)
    static constexpr int SL = SBLOCK + 16 / (int)sizeof(real);     // stage slice: one run + 16 bytes
};
constexpr int QT_THREADS = SBLOCK + 32;         // eight consumer warps and the producer warp
constexpr int QT_HDR = 256;                     // shared-memory header: 2 x 8 mbarriers
constexpr int QT_ERR_BIT = 2;
constexpr long long QT_WAIT_CAP = 1LL << 24;
__device__ __forceinline__ bool mbar_wait_capped(unsigned bar, unsigned parity, long long cap) {
    unsigned done = 0;
    for (long long it = 0; it < cap && !done; ++it)
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return done != 0;
}
template <typename real, bool ENERGY>
__global__ void __launch_bounds__(QT_THREADS, 3) k_qapply_t(const SBlk* __restrict__ blks, const DCls* __restrict__ c1,
                                                            const int2* __restrict__ soff2, SymGeo g, const real* __restrict__ qs,
                                                            const real* __restrict__ ep, real* __restrict__ x, real* __restrict__ xp,
                                                            double2* part, int nst, int* err) {
    constexpr int SPS = QtCfg<real>::SPS, SL = QtCfg<real>::SL, NCW = SBLOCK / 32;
    extern __shared__ __align__(16) unsigned char qt_raw[];
    unsigned long long* full = (unsigned long long*)qt_raw;                       // nst <= 8 each
    unsigned long long* empty = full + 8;
    real* stg = (real*)(qt_raw + QT_HDR);                                         // nst * SPS slices of SL
    int2* s_o2 = (int2*)(qt_raw + QT_HDR + (size_t)nst * SPS * SL * sizeof(real));   // the class's slot offsets
    const SBlk B = blks[blockIdx.x];
    const DCls C = c1[B.cls];
    const int ns = C.st_end - C.st_begin, nup = C.nup, nch = (ns + SPS - 1) / SPS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int s = tid; s < ns; s += blockDim.x) s_o2[s] = soff2[C.st_begin + s];
    if (tid == 0) {
        for (int st = 0; st < nst; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + st)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(empty + st)), "r"(NCW));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const real* qrow = qs + (B.q0 + B.t0);        // slot offset 0 of the block's first lattice point
    const int t = B.t0 + tid;
    const int vy = t / g.NX, vx = t - vy * g.NX;
    const int rx = vx - C.lo[0], ry = vy - C.lo[1];
    const bool row = tid < B.cnt && tid < SBLOCK && (unsigned)rx < (unsigned)C.num[0] && (unsigned)ry < (unsigned)C.num[1];
    const int pe = C.pbase + ((B.vz + g.H) * g.NP + (vy + g.H)) * g.NP + vx + g.H;
    KSum<real> a;
    bool failed = false;
    if (warp == NCW) {
        // producer: stage ch % nst takes chunk ch once the consumers have released chunk ch - nst
        unsigned long long pol;
        int ch = 0;
        for (; ch < nch; ++ch) {
            const int st = ch % nst, s0 = ch * SPS, m = min(SPS, ns - s0);
            if (ch >= nst) {
                const bool ok = lane != 0 || mbar_wait_capped(smem_u32(empty + st), (unsigned)((ch / nst - 1) & 1), QT_WAIT_CAP);
                if (!__all_sync(0xffffffffu, ok)) {
                    failed = true;
                    break;
                }
            }
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(full + st)),
                             "r"((unsigned)(m * SL * (int)sizeof(real)))
                             : "memory");
            __syncwarp();
            if (lane < m) {
                const int s = s0 + lane;
                if (s < nup)
                    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
                else
                    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
                const uintptr_t src = (uintptr_t)(qrow + s_o2[s].x) & ~(uintptr_t)15;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
                        smem_u32(stg + (size_t)(st * SPS + lane) * SL)),
                    "l"(src), "r"((unsigned)(SL * sizeof(real))), "r"(smem_u32(full + st)), "l"(pol)
                    : "memory");
            }
        }
        // copies can be in flight only for the last nst chunks issued (one per stage): the producer
        // waits for them, so that none lands after the block has gone even if a consumer gave up
        if (lane == 0) {
            bool landed = true;
            for (int c = max(0, ch - nst); c < ch; ++c)
                landed &= mbar_wait_capped(smem_u32(full + c % nst), (unsigned)((c / nst) & 1), QT_WAIT_CAP);
            if (failed || !landed) atomicOr(err, QT_ERR_BIT);
        }
        __syncwarp();
    } else {
        const real* __restrict__ e0 = ep + pe;
        for (int ch = 0; ch < nch; ++ch) {
            const int st = ch % nst;
            if (!__all_sync(0xffffffffu, mbar_wait_capped(smem_u32(full + st), (unsigned)((ch / nst) & 1), QT_WAIT_CAP))) {
                if (lane == 0) atomicOr(err, QT_ERR_BIT);
                failed = true;
                break;
            }
            if (row) {
                const real* sq = stg + (size_t)st * SPS * SL;
                const int s0 = ch * SPS;
                real qv[SPS], ev[SPS];
#pragma unroll
                for (int u = 0; u < SPS; ++u) {
                    qv[u] = real(0);
                    ev[u] = real(0);
                    if (s0 + u < ns) {
                        const int2 o = s_o2[s0 + u];
                        const int sh = (int)(((uintptr_t)(qrow + o.x) & 15) / sizeof(real));
                        qv[u] = sq[u * SL + sh + tid];
                        ev[u] = __ldg(e0 + o.y);
                    }
                }
#pragma unroll
                for (int u = 0; u < SPS; ++u)
                    if (s0 + u < ns) a.add(qv[u], ev[u]);
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(empty + st)) : "memory");
        }
    }
    Neu w{0.0, 0.0};
    if (row && !failed) {
        x[C.off + ((long long)(B.vz - C.lo[2]) * C.num[1] + ry) * C.num[0] + rx] = a.s;
        xp[pe] = a.s;
        if (ENERGY) w = neu_add(w, (double)ep[pe] * (double)a.s);
    }
    if (ENERGY) {
        w = block_reduce(w);
        if (threadIdx.x == 0) part[blockIdx.x] = make_double2(w.s, w.c);
    }
}

// partial[blockIdx] = sum_i e_i x_i over a grid-stride slice (fixed order)
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_dot(const real* __restrict__ a, const real* __restrict__ b, long long n,
                                               double2* part) {
    Neu v{0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v = neu_add(v, (double)a[i] * (double)b[i]);
    v = block_reduce(v);
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(v.s, v.c);
}

// partial[blockIdx] = sum_T (1/mu_T) bn_T^T M2a bo_T  (one thread per tet, FP64)
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_tet_quad(Tables tb, const double* __restrict__ M2a, const real* __restrict__ bn,
                                                    const real* __restrict__ bo, const real* __restrict__ inv_mu,
                                                    double2* part) {
    const int n = tb.n, n2a = tb.n2a;
    const long long T = 6LL * n * n * n;
    Neu v{0.0, 0.0};
    double vn[27], vo[27];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t % 6);
        const long long cube = t / 6;
        const int cx = (int)(cube % n), cy = (int)((cube / n) % n), cz = (int)(cube / ((long long)n * n));
        for (int r = 0; r < n2a; ++r) {
            const DLoc2 Lr = tb.loc2[s * n2a + r];
            const DCls D = tb.c2[Lr.cls];
            const int ux = cx + Lr.off[0] - D.lo[0], uy = cy + Lr.off[1] - D.lo[1], uz = cz + Lr.off[2] - D.lo[2];
            if (in_box(D, ux, uy, uz)) {
                const long long g = D.off + ((long long)uz * D.num[1] + uy) * D.num[0] + ux;
                vn[r] = (double)bn[g];
                vo[r] = (double)bo[g];
            } else {
                vn[r] = 0.0;
                vo[r] = 0.0;
            }
        }
        double q = 0.0;
        for (int r = 0; r < n2a; ++r) {
            double u = 0.0;
            for (int c = 0; c < n2a; ++c) u += M2a[r * n2a + c] * vo[c];
            q += vn[r] * u;
        }
        if (inv_mu) q *= (double)inv_mu[t];
        v = neu_add(v, q);
    }
    v = block_reduce(v);
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(v.s, v.c);
}

// W_n of one column in one launch after an ENERGY Q1 apply:
//   out = 1/2 sum(qpart) + 1/2 sum_T (1/mu_T) bn_T^T M2a bo_T
// qpart holds the per-block e_i x_i partials of k_qapply_s.  Each block sums its tets into a
// Neumaier pair (the per-tet product runs in the arithmetic type A: float for FP32 contexts,
// double for FP64); the block that finishes last (ticket counter) merges every partial in
// block order, so the result does not depend on the block schedule, and resets the counter.
template <typename real, typename A>
__global__ void __launch_bounds__(BLOCK) k_tet_energy(Tables tb, const A* __restrict__ M2a, const real* __restrict__ bn,
                                                      const real* __restrict__ bo, const real* __restrict__ inv_mu,
                                                      double2* part, const double2* __restrict__ qpart, int nq,
                                                      unsigned* ticket, double* out) {
    const int n = tb.n, n2a = tb.n2a;
    const long long T = 6LL * n * n * n;
    Neu v{0.0, 0.0};
    A vn[27], vo[27];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x) {
        const int sh = (int)(t % 6);
        const long long cube = t / 6;
        const int cx = (int)(cube % n), cy = (int)((cube / n) % n), cz = (int)(cube / ((long long)n * n));
        for (int r = 0; r < n2a; ++r) {
            const DLoc2 Lr = tb.loc2[sh * n2a + r];
            const DCls D = tb.c2[Lr.cls];
            const int ux = cx + Lr.off[0] - D.lo[0], uy = cy + Lr.off[1] - D.lo[1], uz = cz + Lr.off[2] - D.lo[2];
            if (in_box(D, ux, uy, uz)) {
                const long long gi = D.off + ((long long)uz * D.num[1] + uy) * D.num[0] + ux;
                vn[r] = (A)bn[gi];
                vo[r] = (A)bo[gi];
            } else {
                vn[r] = A(0);
                vo[r] = A(0);
            }
        }
        A q = A(0);
        for (int r = 0; r < n2a; ++r) {
            A u = A(0);
            for (int c = 0; c < n2a; ++c) u = fma(M2a[r * n2a + c], vo[c], u);
            q = fma(vn[r], u, q);
        }
        double qd = (double)q;
        if (inv_mu) qd *= (double)inv_mu[t];
        v = neu_add(v, qd);
    }
    v = block_reduce(v);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = make_double2(v.s, v.c);
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    Neu a{0.0, 0.0}, b{0.0, 0.0};
    for (int i = threadIdx.x; i < nq; i += blockDim.x) a = neu_merge(a, Neu{__ldcg(&qpart[i].x), __ldcg(&qpart[i].y)});
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) b = neu_merge(b, Neu{__ldcg(&part[i].x), __ldcg(&part[i].y)});
    a = block_reduce(a);
    __syncthreads();
    b = block_reduce(b);
    if (threadIdx.x == 0) {
        *out = 0.5 * (a.s + a.c) + 0.5 * (b.s + b.c);
        *ticket = 0u;
    }
}

// out[slot] = 0.5 * (sum of parts1) + 0.5 * (sum of parts2), fixed order, one block
__global__ void k_finish(const double2* __restrict__ p1, int n1, const double2* __restrict__ p2, int n2,
                         double* out) {
    Neu a{0.0, 0.0}, b{0.0, 0.0};
    for (int i = threadIdx.x; i < n1; i += blockDim.x) a = neu_merge(a, Neu{p1[i].x, p1[i].y});
    for (int i = threadIdx.x; i < n2; i += blockDim.x) b = neu_merge(b, Neu{p2[i].x, p2[i].y});
    a = block_reduce(a);
    __syncthreads();
    b = block_reduce(b);
    if (threadIdx.x == 0) *out = 0.5 * (a.s + a.c) + 0.5 * (b.s + b.c);
}

// ---- energies per right-hand side (R > 1): part[block][col], fixed-order merges
// the block's threads with equal column merge their partial sums in thread order
__device__ Neu block_reduce_col(Neu v, int rshift, Neu* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    const int R = 1 << rshift;
    Neu r{0.0, 0.0};
    if ((int)threadIdx.x < R)
        for (int j = threadIdx.x; j < (int)blockDim.x; j += R) r = neu_merge(r, sh[j]);
    __syncthreads();
    return r;
}
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_dot_r(const real* __restrict__ a, const real* __restrict__ b, long long n,
                                                 int rshift, double2* part) {
    __shared__ Neu sh[BLOCK];
    const int R = 1 << rshift, col = threadIdx.x & (R - 1);
    const long long per = blockDim.x >> rshift;
    Neu v{0.0, 0.0};
    for (long long i = (long long)blockIdx.x * per + (threadIdx.x >> rshift); i < n; i += (long long)gridDim.x * per)
        v = neu_add(v, (double)a[(i << rshift) + col] * (double)b[(i << rshift) + col]);
    v = block_reduce_col(v, rshift, sh);
    if ((int)threadIdx.x < R) part[(long long)blockIdx.x * R + threadIdx.x] = make_double2(v.s, v.c);
}
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_tet_quad_r(Tables tb, const double* __restrict__ M2a, const real* __restrict__ bn,
                                                      const real* __restrict__ bo, const real* __restrict__ inv_mu, int rshift,
                                                      double2* part) {
    __shared__ Neu sh[BLOCK];
    const int n = tb.n, n2a = tb.n2a;
    const long long T = 6LL * n * n * n;
    const int R = 1 << rshift, col = threadIdx.x & (R - 1);
    const long long per = blockDim.x >> rshift;
    Neu v{0.0, 0.0};
    double vn[27], vo[27];
    for (long long t = (long long)blockIdx.x * per + (threadIdx.x >> rshift); t < T; t += (long long)gridDim.x * per) {
        const int s = (int)(t % 6);
        const long long cube = t / 6;
        const int cx = (int)(cube % n), cy = (int)((cube / n) % n), cz = (int)(cube / ((long long)n * n));
        for (int r = 0; r < n2a; ++r) {
            const DLoc2 Lr = tb.loc2[s * n2a + r];
            const DCls D = tb.c2[Lr.cls];
            const int ux = cx + Lr.off[0] - D.lo[0], uy = cy + Lr.off[1] - D.lo[1], uz = cz + Lr.off[2] - D.lo[2];
            if (in_box(D, ux, uy, uz)) {
                const long long gi = ((D.off + ((long long)uz * D.num[1] + uy) * D.num[0] + ux) << rshift) + col;
                vn[r] = (double)bn[gi];
                vo[r] = (double)bo[gi];
            } else {
                vn[r] = 0.0;
                vo[r] = 0.0;
            }
        }
        double q = 0.0;
        for (int r = 0; r < n2a; ++r) {
            double u = 0.0;
            for (int c = 0; c < n2a; ++c) u += M2a[r * n2a + c] * vo[c];
            q += vn[r] * u;
        }
        if (inv_mu) q *= (double)inv_mu[t];
        v = neu_add(v, q);
    }
    v = block_reduce_col(v, rshift, sh);
    if ((int)threadIdx.x < R) part[(long long)blockIdx.x * R + threadIdx.x] = make_double2(v.s, v.c);
}
// out[col] = 0.5 sum_blocks p1[block][col] + 0.5 sum_blocks p2[block][col], one thread per column
__global__ void k_finish_r(const double2* __restrict__ p1, const double2* __restrict__ p2, int nblk, int R, double* out) {
    for (int col = threadIdx.x; col < R; col += blockDim.x) {
        Neu a{0.0, 0.0}, b{0.0, 0.0};
        for (int i = 0; i < nblk; ++i) {
            a = neu_merge(a, Neu{p1[(long long)i * R + col].x, p1[(long long)i * R + col].y});
            b = neu_merge(b, Neu{p2[(long long)i * R + col].x, p2[(long long)i * R + col].y});
        }
        out[col] = 0.5 * (a.s + a.c) + 0.5 * (b.s + b.c);
    }
}

// ------------------------------------------------------------------ e += ctau C^T M2 b on tensor cores (R >= 32 columns)
// With a uniform permeability C^T M2 is one constant stencil per 1-form class (the merged weights).
// Over the union U of the (2-form class, offset) terms of every curl-carrying class it is a dense
// matrix W (classes x K), the same at every lattice point, so for a batch of P lattice points
// (P R = 128 rows) the update of all classes is one GEMM with a shared operand:
//     D[(p, r), j] = sum_k Bg[(p, r), k] W[j, k],   Bg[(p, r), k] = b[(U_k at v_p), r]
// run as tcgen05.mma kind::tf32 with M = 128 (rows = point x column), N = classes (padded to 16),
// K = |U| (padded to 8), D in tensor memory, FP32 accumulation.  A (the gathered b) and B (W^T)
// are K-major, no swizzle: core matrices of 8 rows x 16 bytes, element (m, k) at byte
//     (m / 8) SBO + (k / 4) * 128 + (m % 8) * 16 + (k % 4) * 4,
// SBO = 128 K/4 + 16 (the extra 16 bytes put the 8-row groups on different banks so that the
// transposing gather writes without conflicts).  PASSES = 1: TF32 operands (truncated by the
// tensor core); PASSES = 3: each operand split as hi + lo with hi = its TF32 part, and
// D = Ahi Bhi + Ahi Blo + Alo Bhi (about 2^-21 relative per product, FP32 level).
// One elected thread issues the MMAs; completion is signalled on an mbarrier whose wait has an
// iteration cap: on timeout the kernel sets *err and stops (after freeing its tensor memory).
struct TcGeo {
    int n, rshift, P;            // cubes per side, log2 R, lattice points per batch (P R = 128)
    int nbatch;                  // ceil(n^3 / P)
    int Kp, Nc, Ma;              // padded K, padded N, curl-carrying 1-form classes
    int sboA, sboB;              // 8-row group strides (bytes)
    int offAlo, offBhi, offBlo, offIdx, offBar;   // shared-memory layout (bytes from the 1024-aligned base)
    int tmem_cols;
};
__device__ __forceinline__ unsigned long long umma_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // version 1, no swizzle
}
__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }
// 3xTF32 tables fill most of shared memory (one CTA per SM): 16 warps, all of which gather.  One
// pass: 8 warps, so that two CTAs fit per SM.  Warps 0-7 read the accumulator back (4 lane
// quarters x 2 column halves).
template <int PASSES>
constexpr int tc_threads() { return PASSES == 3 ? 512 : 256; }
template <int PASSES>
__global__ void __launch_bounds__(tc_threads<PASSES>(), 1) k_curlT_e_tc(TcGeo G, const int4* __restrict__ uterm, const DCls* __restrict__ c1,
                                                       const DCls* __restrict__ c2, const int* __restrict__ acls,
                                                       const float* __restrict__ Wt, const float* __restrict__ b,
                                                       float* __restrict__ e, float* __restrict__ ep, PadGeo pg,
                                                       Tau<float> ctau, int* __restrict__ err) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sAhi = sm;
    unsigned char* sAlo = sm + G.offAlo;
    unsigned char* sBhi = sm + G.offBhi;
    unsigned char* sBlo = sm + G.offBlo;
    int* gidx = (int*)(sm + G.offIdx);                      // [P][Kp] compact 2-form index or -1
    unsigned long long* bar = (unsigned long long*)(sm + G.offBar);
    unsigned* tslot = (unsigned*)(sm + G.offBar + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = 1 << G.rshift, KC = G.Kp >> 2;
    // B = W^T (N x K, K-major), hi (and lo) parts, once per CTA
    for (int i = tid; i < G.Nc * G.Kp; i += blockDim.x) {
        const int nrow = i / G.Kp, k = i - nrow * G.Kp;
        const float w = Wt[i];
        const int off = (nrow >> 3) * G.sboB + (k >> 2) * 128 + (nrow & 7) * 16 + (k & 3) * 4;
        const float hi = PASSES == 3 ? tf32_hi(w) : w;
        *(float*)(sBhi + off) = hi;
        if (PASSES == 3) *(float*)(sBlo + off) = w - hi;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"((unsigned)G.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = *tslot;
    // instruction descriptor: D f32, A/B tf32, K-major both, N >> 3, M = 128 >> 4
    const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(G.Nc >> 3) << 17) | ((128u >> 4) << 24);
    const int n = G.n, n3 = n * n * n;
    unsigned phase = 0;
    bool failed = false;
    for (int bt = blockIdx.x; bt < G.nbatch && !failed; bt += gridDim.x) {
        // 2-form indices of the union terms at the batch's points
        for (int i = tid; i < G.P * G.Kp; i += blockDim.x) {
            const int p = i / G.Kp, k = i - p * G.Kp;
            const int pt = bt * G.P + p;
            int gi = -1;
            const int4 U = uterm[k];
            if (pt < n3 && U.x >= 0) {
                const int vx = pt % n, vy = (pt / n) % n, vz = pt / (n * n);
                const DCls D = c2[U.x];
                const int ux = vx + U.y - D.lo[0], uy = vy + U.z - D.lo[1], uz = vz + U.w - D.lo[2];
                if (in_box(D, ux, uy, uz)) gi = (int)(D.off + ((long long)uz * D.num[1] + uy) * D.num[0] + ux);
            }
            gidx[i] = gi;
        }
        __syncthreads();
        // A = gathered b, K-major: one warp instruction fills an (8 rows x 4 k) tile, conflict-free;
        // eight tiles per round, their loads issued before the first store
        {
            const int nw = blockDim.x >> 5, ntile = 16 * KC;
            for (int t0 = warp; t0 < ntile; t0 += 8 * nw) {
                float v[8];
                int off[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int tile = t0 + u * nw;
                    v[u] = 0.f;
                    off[u] = -1;
                    if (tile < ntile) {
                        const int grp = tile / KC, kc = tile - grp * KC;
                        const int m = grp * 8 + (lane & 7), k = kc * 4 + (lane >> 3);
                        const int p = m >> G.rshift, r = m & (R - 1);
                        const int gi = p < G.P ? gidx[p * G.Kp + k] : -1;
                        if (gi >= 0) v[u] = __ldg(b + ((long long)gi << G.rshift) + r);
                        off[u] = grp * G.sboA + kc * 128 + (lane & 7) * 16 + (lane >> 3) * 4;
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (off[u] >= 0) {
                        const float hi = PASSES == 3 ? tf32_hi(v[u]) : v[u];
                        *(float*)(sAhi + off[u]) = hi;
                        if (PASSES == 3) *(float*)(sAlo + off[u]) = v[u] - hi;
                    }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int ks = 0; ks < (G.Kp >> 3); ++ks) {
                const unsigned long long ahi = umma_desc(smem_u32(sAhi) + ks * 256, 128, G.sboA);
                const unsigned long long bhi = umma_desc(smem_u32(sBhi) + ks * 256, 128, G.sboB);
                const unsigned acc = ks > 0 ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                             "l"(ahi), "l"(bhi), "r"(idesc), "r"(acc));
                if (PASSES == 3) {
                    const unsigned long long alo = umma_desc(smem_u32(sAlo) + ks * 256, 128, G.sboA);
                    const unsigned long long blo = umma_desc(smem_u32(sBlo) + ks * 256, 128, G.sboB);
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                                 "l"(ahi), "l"(blo), "r"(idesc), "r"(1u));
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                                 "l"(alo), "l"(bhi), "r"(idesc), "r"(1u));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
        }
        // wait for the MMAs (bounded)
        {
            unsigned done = 0;
            for (long long it = 0; it < (1LL << 26) && !done; ++it)
                asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
                             : "=r"(done)
                             : "r"(smem_u32(bar)), "r"(phase));
            failed = __syncthreads_or(!done) != 0;     // the same decision in every thread
            if (failed && tid == 0) atomicOr(err, 1);
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!failed && warp < 8) {
            // epilogue: warp w < 8 reads lanes 32 (w % 4) .. +31 (rows m) and half of the columns
            const int m = (warp & 3) * 32 + lane;
            const int p = m >> G.rshift, r = m & (R - 1);
            const int pt = bt * G.P + p;
            const bool okp = p < G.P && pt < n3;
            const int vx = pt % n, vy = (pt / n) % n, vz = pt / (n * n);
            const int half = G.Nc >> 1, j0 = (warp >> 2) * half;
            for (int jc = j0; jc < j0 + half; jc += 8) {
                unsigned v[8];
                const unsigned taddr = tmem + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)jc;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (!okp) continue;
                long long gi[8], pi[8];
                float eo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = jc + u;
                    gi[u] = -1;
                    pi[u] = 0;
                    eo[u] = 0.f;
                    if (j < G.Ma) {
                        const DCls C = c1[acls[j]];
                        const int rx = vx - C.lo[0], ry = vy - C.lo[1], rz = vz - C.lo[2];
                        if (in_box(C, rx, ry, rz)) {
                            gi[u] = ((C.off + ((long long)rz * C.num[1] + ry) * C.num[0] + rx) << G.rshift) + r;
                            pi[u] = ((long long)pad_index(C, pg, vx, vy, vz) << G.rshift) + r;
                            eo[u] = e[gi[u]];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (gi[u] >= 0) {
                        const float d = __uint_as_float(v[u]);
                        const float nv = fmaf(ctau.lo, d, fmaf(ctau.hi, d, eo[u]));
                        e[gi[u]] = nv;
                        ep[pi[u]] = nv;
                    }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)G.tmem_cols));
}

// ------------------------------------------------------------------ uneven batch: many cavities, one launch
// Independent cavities of any size and order, each with its own tables, Q1 and state, step
// together in one persistent launch.  A step is three phases over work items (cavity, block):
//   A  x = Q1 e (curl-carrying rows)     B  b_{n+1/2} = b_{n-1/2} - dt C x     C  e += dt C^T M2 b - j
// with a grid-wide barrier after each.  The item bodies are the ones of the one-column lattice
// kernels; a cavity's blocks only touch that cavity's buffers.  The barrier spins with an
// iteration cap: when it is reached the kernel sets *err and every CTA leaves at the next
// barrier, so a missing CTA can stall the launch for a bounded time only.
template <typename real>
struct BCav {
    const DCls *c1, *c2;
    const int2* soff2;
    SymGeo sg;
    PadGeo pg;
    const real* qs;
    real *ep, *x, *xp, *bp, *b0, *b1, *e;
    const CTermL* cterms;
    const int* pbeg;
    const WTermL<real>* wterms;
    const SBlk *blkA, *blkB, *blkC;
    const int* sbeg;                 // source entries of blkC (NULL: no source)
    const SrcE<real>* sent;
    Tau<real> tau;
    int cur0;                        // b ping-pong index at the first step of the launch
};
template <typename real>
__device__ __forceinline__ void qapply_rows(const SBlk& B, const DCls& C, const int2* s_o2, SymGeo g, const real* __restrict__ qs,
                                            const real* __restrict__ ep, real* __restrict__ x, real* __restrict__ xp) {
    if ((int)threadIdx.x >= B.cnt) return;
    const int t = B.t0 + (int)threadIdx.x;
    const int vy = t / g.NX, vx = t - vy * g.NX;
    const int rx = vx - C.lo[0], ry = vy - C.lo[1];
    if ((unsigned)rx >= (unsigned)C.num[0] || (unsigned)ry >= (unsigned)C.num[1]) return;
    unsigned long long keep, drop;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(drop));
    const real* __restrict__ q = qs + (B.q0 + t);
    const int pe = C.pbase + ((B.vz + g.H) * g.NP + (vy + g.H)) * g.NP + vx + g.H;
    const real* __restrict__ e0 = ep + pe;
    KSum<real> a;
    qs_run(a, s_o2, 0, C.nup, q, e0, keep);
    qs_run(a, s_o2, C.nup, C.st_end - C.st_begin, q, e0, drop);
    x[C.off + ((long long)(B.vz - C.lo[2]) * C.num[1] + ry) * C.num[0] + rx] = a.s;
    xp[pe] = a.s;
}
// grid-wide barrier over a co-resident grid (bar[0] arrivals, bar[1] generation); returns false
// in every thread of every CTA once any CTA gave up waiting
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen, int* err, int* s_flag, long long cap) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g = gen;
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], g + 1u);
        } else {
            long long it = 0;
            unsigned cur;
            do {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&bar[1]));
                if (cur != g) break;
                __nanosleep(128);
            } while (++it < cap);
            if (cur == g) atomicExch(err, 1);
        }
        __threadfence();
        *s_flag = *(volatile int*)err;
    }
    __syncthreads();
    ++gen;
    return *s_flag == 0;
}
template <typename real>
__global__ void __launch_bounds__(SBLOCK) k_batch(const BCav<real>* __restrict__ cavs, const int2* __restrict__ items, int nA,
                                                  int nB, int nC, int nsteps, int ncav, const double* __restrict__ amp,
                                                  unsigned* bar, int* err, long long cap) {
    extern __shared__ __align__(16) unsigned char braw[];
    int2* s_o2 = reinterpret_cast<int2*>(braw);
    WTermL<real>* s_t = reinterpret_cast<WTermL<real>*>(braw);
    __shared__ int s_flag;
    __shared__ unsigned s_gen;
    if (threadIdx.x == 0) asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(s_gen) : "l"(&bar[1]));
    __syncthreads();
    unsigned gen = s_gen;
    const int2* iA = items;
    const int2* iB = items + nA;
    const int2* iC = items + nA + nB;
    for (int st = 0; st < nsteps; ++st) {
        for (int i = blockIdx.x; i < nA; i += gridDim.x) {
            const int2 it = iA[i];
            const BCav<real>& cv = cavs[it.x];
            const SBlk B = cv.blkA[it.y];
            const DCls C = cv.c1[B.cls];
            __syncthreads();
            for (int s = threadIdx.x; s < C.st_end - C.st_begin; s += blockDim.x) s_o2[s] = cv.soff2[C.st_begin + s];
            __syncthreads();
            qapply_rows(B, C, s_o2, cv.sg, cv.qs, cv.ep, cv.x, cv.xp);
        }
        if (!grid_barrier(bar, gen, err, &s_flag, cap)) return;
        for (int i = blockIdx.x; i < nB; i += gridDim.x) {
            const int2 it = iB[i];
            const BCav<real>& cv = cavs[it.x];
            const bool odd = ((cv.cur0 + st) & 1) != 0;
            curl_b_rows(cv.blkB[it.y], cv.c2, cv.cterms, cv.pg, cv.sg.NX, cv.xp, odd ? cv.b1 : cv.b0, odd ? cv.b0 : cv.b1,
                        cv.bp, cv.tau);
        }
        if (!grid_barrier(bar, gen, err, &s_flag, cap)) return;
        for (int i = blockIdx.x; i < nC; i += gridDim.x) {
            const int2 it = iC[i];
            const BCav<real>& cv = cavs[it.x];
            const SBlk B = cv.blkC[it.y];
            const int tb = cv.pbeg[B.cls], nt = cv.pbeg[B.cls + 1] - tb;
            __syncthreads();
            for (int s = threadIdx.x; s < nt; s += blockDim.x) s_t[s] = cv.wterms[tb + s];
            __syncthreads();
            const double* a = cv.sbeg ? amp + (long long)st * ncav + it.x : nullptr;
            curlT_e_rows(B, cv.c1, s_t, nt, cv.pg, cv.sg.NX, cv.bp, cv.e, cv.tau, cv.ep, cv.sbeg, cv.sent, a, it.y);
        }
        if (!grid_barrier(bar, gen, err, &s_flag, cap)) return;
    }
}

// ------------------------------------------------------------------ adjoint of the leapfrog (one column)
// The reverse sweep of the probe-region energy
//     L = tau sum_n [1/2 x_n^T M1^R x_n + 1/2 b_{n+1/2}^T M2^R b_{n+1/2}],  x_n = Q1 e_n,
// runs the transposed shear maps newest step first.  With cb = C^T bbar (bbar itself is never
// needed) one reverse step is
//     cb   += tau C^T M2 (C ebar) + tau C^T M2^R b_{n+1/2}
//     xbar  = -tau cb + tau M1^R x_n
//     ebar += Q1 xbar,      Q1bar += xbar e_n^T
// C ebar and C^T M2 u reuse k_curl_b_s / k_curlT_e_s, Q1 xbar reuses k_qapply_s.  The kernels below
// are the rest: the region operators (CSR over the DoFs of the region's tets), the Q1bar
// accumulation on the upper-triangle lattice of Q1, and the per-tet loss / M1^R gradient terms.

// y[rows[i]] += alpha sum_k val[k] x[col[k]] (one thread per listed row)
template <typename real>
__global__ void k_csr_add(int nrows, const int* __restrict__ rows, const int* __restrict__ ptr, const int* __restrict__ col,
                          const double* __restrict__ val, const real* __restrict__ x, real* __restrict__ y, double alpha) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    double a = 0.0;
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) a += val[k] * (double)x[col[k]];
    y[rows[i]] = (real)((double)y[rows[i]] + alpha * a);
}
// xbar (padded) = -tau cb + tau (M1^R x); M1^R as a CSR over every 1-form row (most rows empty)
template <typename real>
__global__ void k_xbar(long long N1, const int* __restrict__ pidx, const int* __restrict__ ptr, const int* __restrict__ col,
                       const double* __restrict__ val, const real* __restrict__ cb, const real* __restrict__ x, double tau,
                       real* __restrict__ xbar_pad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N1; i += (long long)gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) m += val[k] * (double)x[col[k]];
        xbar_pad[pidx[i]] = (real)(tau * (m - (double)cb[i]));
    }
}
// a += b over a padded vector (halo entries are zero in both)
template <typename real>
__global__ void k_pad_add(long long n, real* __restrict__ a, const real* __restrict__ b) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] += b[i];
}
// Q1bar on the stored (upper) pairs: S[i, s] += xbar_i e_j + xbar_j e_i, j = the slot's neighbour.
// Same blocks, slot tables and padded geometry as k_qapply_s; the upper slots are the first C.nup
// of the class's slot list.  One thread owns each stored value: no atomics.
template <typename real>
__global__ void __launch_bounds__(SBLOCK) k_q1bar(const SBlk* __restrict__ blks, const DCls* __restrict__ c1,
                                                  const int2* __restrict__ soff2, SymGeo g, const real* __restrict__ xb,
                                                  const real* __restrict__ ep, real* __restrict__ S) {
    extern __shared__ __align__(16) int2 s_o2[];
    const SBlk B = blks[blockIdx.x];
    const DCls C = c1[B.cls];
    for (int s = threadIdx.x; s < C.nup; s += blockDim.x) s_o2[s] = soff2[C.st_begin + s];
    __syncthreads();
    if ((int)threadIdx.x >= B.cnt) return;
    const int t = B.t0 + (int)threadIdx.x;
    const int vy = t / g.NX, vx = t - vy * g.NX;
    const int rx = vx - C.lo[0], ry = vy - C.lo[1];
    if ((unsigned)rx >= (unsigned)C.num[0] || (unsigned)ry >= (unsigned)C.num[1]) return;
    const int pe = C.pbase + ((B.vz + g.H) * g.NP + (vy + g.H)) * g.NP + vx + g.H;
    const real xi = xb[pe], ei = ep[pe];
    real* __restrict__ q = S + (B.q0 + t);
    for (int s = 0; s < C.nup; ++s) {
        const int2 o = s_o2[s];
        q[o.x] += xi * ep[pe + o.y] + xb[pe + o.y] * ei;
    }
}
// Region tets (one thread each): loss[t] += tau (eps_t/2 x_T^T M1 x_T + 1/(2 mu_t) b_T^T M2a b_T) and
// grad[t] += tau/2 x_T^T M1 x_T, in FP64, from the unweighted local blocks.
template <typename real>
__global__ void k_region(int nt, int n1, int n2a, const int* __restrict__ d1, const int* __restrict__ d2,
                         const double* __restrict__ M1l, const double* __restrict__ M2l, const double* __restrict__ epsr,
                         const double* __restrict__ imur, const real* __restrict__ x, const real* __restrict__ b,
                         double tau, double* __restrict__ loss, double* __restrict__ grad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double xv[45], bv[36];
    for (int a = 0; a < n1; ++a) {
        const int i = d1[(long long)t * n1 + a];
        xv[a] = i >= 0 ? (double)x[i] : 0.0;
    }
    for (int a = 0; a < n2a; ++a) {
        const int i = d2[(long long)t * n2a + a];
        bv[a] = i >= 0 ? (double)b[i] : 0.0;
    }
    double qx = 0.0, qb = 0.0;
    for (int a = 0; a < n1; ++a) {
        double u = 0.0;
        for (int c = 0; c < n1; ++c) u += M1l[a * n1 + c] * xv[c];
        qx += xv[a] * u;
    }
    for (int a = 0; a < n2a; ++a) {
        double u = 0.0;
        for (int c = 0; c < n2a; ++c) u += M2l[a * n2a + c] * bv[c];
        qb += bv[a] * u;
    }
    loss[t] += tau * (0.5 * epsr[t] * qx + 0.5 * imur[t] * qb);
    grad[t] += 0.5 * tau * qx;
}

}  // namespace

// ====================================================================== context
struct ygm_ctx {
    ygm::Setup S;
    int precision = YGM_FP64, n_rhs = 1, rshift = 0, energy_every = 0, device = 0;   // n_rhs = 2^rshift
    size_t rs = 8;                          // sizeof(real)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device memory
    void *e = nullptr, *b[2] = {nullptr, nullptr}, *x = nullptr, *bscr = nullptr, *q = nullptr;
    void *W = nullptr, *inv_mu = nullptr, *sw = nullptr;
    double* M2a = nullptr;
    DCls *c1 = nullptr, *c2 = nullptr;
    DSlot* slots = nullptr;
    DTerm* terms = nullptr;
    DInc* inc = nullptr;
    DLoc2* loc2 = nullptr;
    DRow* rowsE = nullptr;
    int nrowsE = 0;
    double2* part = nullptr;
    int npart = 0;
    double* hist = nullptr;
    int64_t hist_cap = 0, hist_n = 0;
    DSrc* dsrc = nullptr;
    long long* sdofs = nullptr;
    int nsrc = 0, nsrc_cap = 0, nsw_cap = 0;
    std::vector<ygm_source> src_cache;
    double* damp[2] = {nullptr, nullptr};    // per-step source amplitudes, double-buffered
    double* hamp[2] = {nullptr, nullptr};    // pinned host staging of the same
    size_t damp_cap[2] = {0, 0};
    cudaEvent_t damp_ev[2] = {nullptr, nullptr};
    int damp_cur = 0;
    // tiled kernels
    QSlot* qslots = nullptr;
    QBlock* qblocks = nullptr;
    int nqblocks = 0, max_slots = 0, qthreads = BLOCK;
    QBlock *eblocks = nullptr, *bblocks = nullptr;
    int neblocks = 0, nbblocks = 0, max_terms = 0;
    // padded copy of e and full-row Q1 (k_qapply_p)
    void *ep = nullptr, *qf = nullptr;
    PBlk* pblks = nullptr;                   // every row of every class (first npblks_act: curl-carrying rows)
    int npblks = 0, npblks_act = 0, max_ns = 0;
    int* soff = nullptr;
    int2* planes = nullptr;                  // (class, vz) of every non-empty 1-form plane
    int nplanes = 0;
    PadGeo pg{0, 0};
    long long n1pad = 0;
    int* spdofs = nullptr;                   // padded indices of the source DoFs
    // upper-triangle Q1 on the anchor lattice (k_qapply_s, one column)
    bool use_sym = false;
    void* qsd = nullptr;
    int2* soff2 = nullptr;
    SBlk* sblks = nullptr;                   // [curl-carrying classes, z-plane order][all classes, z-plane order]
    int nsblks_act = 0, nsblks_all = 0;
    SymGeo sg{0, 0, 0};
    // padded x and b with the lattice curl kernels (one column, with k_qapply_s)
    void *xp = nullptr, *bp = nullptr, *wterms = nullptr;
    CTermL* cterms = nullptr;
    SBlk *lblks_b = nullptr, *lblks_e = nullptr;
    int nlb = 0, nle = 0;
    int64_t qc_rows[2] = {0, 0}, qc_unique[2] = {0, 0}, qc_stored[2] = {0, 0};   // [active only, all rows]
    std::vector<double> split_w{1.0};        // weights of the composed splitting (Strang: {1})
    int tc_passes = 0;                       // > 0: C^T M2 on tensor cores (YGM_FP32_TC_*), 1 or 3 TF32 passes
    TcGeo tcg{};
    int4* uterm = nullptr;                   // union of the merged C^T M2 terms (class, dx, dy, dz)
    int* acls = nullptr;                     // curl-carrying 1-form class of each GEMM column
    float* wt = nullptr;                     // merged weights, [column][K]
    bool pdl = true;                         // programmatic dependent launch between the step's kernels
    bool qt_ok = false;                      // k_qapply_t usable (every copied run inside qsym)
    int qt_mode = 0;                         // 0 automatic (k_qapply_s), 1 k_qapply_s, 2 k_qapply_t
    int qt_nst = 0;                          // k_qapply_t stages
    size_t qt_smem = 0;
    int* dev_err = nullptr;                  // bit 1: a k_curlT_e_tc MMA wait timed out; bit QT_ERR_BIT:
                                             // a k_qapply_t copy wait timed out
    size_t tc_smem = 0;
    int tc_grid = 0;
    double2* qpart = nullptr;                // per-block e_i x_i partials of an all-rows k_qapply_s
    unsigned* ticket = nullptr;              // last-block counter of k_tet_energy (kept at 0 between launches)
    void* M2af = nullptr;                    // M2a in the context precision (k_tet_energy)
    std::vector<SBlk> h_lblks_e;             // host copy of lblks_e
    SBlk* lblks_es = nullptr;                // lblks_e + the blocks of curl-free classes holding a source DoF
    int nle_src = 0;
    int* sbeg = nullptr;                     // per block of lblks_es: first source entry
    void* sent = nullptr;                    // SrcE<real> entries
    void* pterms = nullptr;                  // PTerm<real> merged C^T M2 stencil (uniform mu)
    int* pbeg = nullptr;
    // time state
    int cur = 0;
    bool staggered = false;
    int64_t step = 0;
    int64_t step_base = 0;                  // step index where the current dt took over
    double t_base = 0.0;                    // time at step_base
    double dt_prev = 0.0;
    bool host_only = false;
    int64_t launches = 0;
    std::string err;
    Tables tb{};
    // optional per-launch CUDA-event timing (ygm_kernel_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> ev_rec;   // (kernel kind, index of the start event)
};

enum { KQ = 0, KB = 1, KE = 2, KS = 3, KW = 4, NKIND = 5 };

static void time_begin(ygm_ctx* ctx, int kind) {
    if (!ctx->timing) return;
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) {
            ctx->timing = false;
            return;
        }
        ctx->ev_pool.push_back(ev);
    }
    ctx->ev_rec.push_back({kind, ctx->ev_used});
    cudaEventRecord(ctx->ev_pool[ctx->ev_used], ctx->stream);
    ctx->ev_used += 2;
}
static void time_end(ygm_ctx* ctx) {
    if (!ctx->timing || ctx->ev_rec.empty()) return;
    cudaEventRecord(ctx->ev_pool[ctx->ev_rec.back().second + 1], ctx->stream);
}

static std::string g_create_err;
static std::mutex g_err_mutex;
// largest dynamic shared memory each block kernel has been opted in to, per (device, precision):
// cudaFuncSetAttribute applies to the current device only, and the limit is only ever raised
// (a smaller value set by one context would make another context's launches invalid)
static std::mutex g_smem_mutex;
static std::map<std::pair<int, int>, size_t> g_smem_q, g_smem_e;
static size_t& smem_limit(std::map<std::pair<int, int>, size_t>& m, int dev, int prec) {
    auto it = m.find({dev, prec});
    if (it == m.end()) it = m.emplace(std::make_pair(dev, prec), (size_t)48 * 1024).first;
    return it->second;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess) {                                                                   \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(_e);                         \
            return YGM_ECUDA;                                                                      \
        }                                                                                          \
    } while (0)

static int fail(ygm_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

template <typename T>
static int upload(ygm_ctx* ctx, T** dst, const std::vector<T>& v) {
    if (v.empty()) {
        *dst = nullptr;
        return 0;
    }
    CK(cudaMalloc((void**)dst, v.size() * sizeof(T)));
    CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return 0;
}

// upload FP64 host data in the context precision
static int upload_real(ygm_ctx* ctx, void** dst, const std::vector<double>& v) {
    if (v.empty()) {
        *dst = nullptr;
        return 0;
    }
    CK(cudaMalloc(dst, v.size() * ctx->rs));
    if (ctx->precision == YGM_FP64) {
        CK(cudaMemcpy(*dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(v.begin(), v.end());
        CK(cudaMemcpy(*dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    }
    return 0;
}

static std::vector<DRow> make_rows(const std::vector<ygm::DofClass>& cls, int n, bool active_only) {
    // z-slab-major order over all classes: rows of neighbouring slabs stay close in time,
    // so the transposed Q1 reads of k_qapply hit L2.
    std::vector<DRow> rows;
    for (int vz = 0; vz < n; ++vz)
        for (int vy = 0; vy < n; ++vy)
            for (int c = 0; c < (int)cls.size(); ++c) {
                const auto& b = cls[c].box;
                if (active_only && !cls[c].active) continue;
                int ry = vy - b.lo[1], rz = vz - b.lo[2];
                if (ry < 0 || rz < 0 || ry >= b.num[1] || rz >= b.num[2]) continue;
                rows.push_back(DRow{c, vy, vz, (rz * b.num[1] + ry) * b.num[0]});
            }
    return rows;
}

// The device word the kernels set when a bounded wait gives up (read by check_device_flags).
static int alloc_dev_err(ygm_ctx* ctx) {
    if (ctx->dev_err) return 0;
    CK(cudaMalloc((void**)&ctx->dev_err, sizeof(int)));
    CK(cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), ctx->stream));
    return 0;
}

// k_qapply_t stage count: stages = 0 takes the most that fit beside the slot table in 227 KB (at
// most 4: three blocks per SM in FP32), else 2..8 if they fit.  Sets the kernels' shared-memory
// size and asks for the largest shared-memory carveout (the stages, not L1, hold the Q1 stream);
// *bps receives the resident blocks per SM.
static int qt_configure(ygm_ctx* ctx, int stages, int* bps) {
    const bool f64 = ctx->precision == YGM_FP64;
    const size_t slice = (size_t)(f64 ? QtCfg<double>::SPS * QtCfg<double>::SL * 8 : QtCfg<float>::SPS * QtCfg<float>::SL * 4);
    const size_t tab = (size_t)ctx->max_ns * sizeof(int2);
    auto fits = [&](int nst) { return QT_HDR + nst * slice + tab <= 227 * 1024; };
    int nst = 0;
    if (stages == 0) {
        for (int t = 4; t >= 2 && !nst; --t)
            if (fits(t)) nst = t;
        if (!nst) return fail(ctx, YGM_EINVAL, "k_qapply_t: two stages do not fit in shared memory");
    } else {
        if (stages < 2 || stages > 8 || !fits(stages))
            return fail(ctx, YGM_EINVAL, "k_qapply_t: stages must be 2..8 and fit in 227 KB of shared memory");
        nst = stages;
    }
    const size_t smem = QT_HDR + nst * slice + tab;
    const void* ks[2] = {f64 ? (const void*)k_qapply_t<double, false> : (const void*)k_qapply_t<float, false>,
                         f64 ? (const void*)k_qapply_t<double, true> : (const void*)k_qapply_t<float, true>};
    for (const void* k : ks) {
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared));
    }
    ctx->qt_nst = nst;
    ctx->qt_smem = smem;
    if (bps) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, ks[0], QT_THREADS, smem));
    return 0;
}

// k_qapply_s tables (one column only): (Q1, padded e) offsets per stencil slot and the z-plane
// ordered block lists -- curl-carrying classes only, then every class.  Skipped (the full-row
// kernel is used) when the lattice offsets do not fit 32 bits.
static int setup_sym(ygm_ctx* ctx, const std::vector<int>& eoff) {
    ygm::Setup& S = ctx->S;
    ygm::Lattice& L = S.L;
    ctx->use_sym = false;
    if (ctx->n_rhs != 1 || S.qsym.empty() || (size_t)(ctx->max_ns + 8) * sizeof(int2) > 48 * 1024) return 0;
    const int NX = S.qs_nx, NY = S.qs_ny;
    std::vector<int2> o2(S.st_slots.size());
    for (size_t c = 0; c < L.c1.size(); ++c)
        for (int sidx = S.st_begin[c]; sidx < S.st_begin[c + 1]; ++sidx) {
            const auto& st = S.st_slots[sidx];
            long long qo = st.upper ? (long long)st.slot * S.qs_vol
                                    : S.qs_base[st.cls] - S.qs_base[c] + (long long)st.slot * S.qs_vol +
                                          ((long long)st.d[2] * NY + st.d[1]) * NX + st.d[0];
            if (qo > INT32_MAX || qo < INT32_MIN) return 0;
            o2[sidx] = make_int2((int)qo, eoff[sidx]);
        }
    // per class: the upper slots, then the lower ones (k_qapply_s gives the two groups different
    // L2 eviction hints), each group in padded-e order (neighbour class, dz, dy, dx) so that
    // consecutive slots read neighbouring e values, which the L1 then serves
    for (size_t c = 0; c < L.c1.size(); ++c) {
        const int b0 = S.st_begin[c], b1 = S.st_begin[c + 1];
        std::vector<int> idx(b1 - b0);
        for (int i = 0; i < b1 - b0; ++i) idx[i] = b0 + i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            const int ua = S.st_slots[a].upper ? 0 : 1, ub = S.st_slots[b].upper ? 0 : 1;
            return ua != ub ? ua < ub : o2[a].y < o2[b].y;
        });
        std::vector<int2> sorted(b1 - b0);
        for (int i = 0; i < b1 - b0; ++i) sorted[i] = o2[idx[i]];
        std::copy(sorted.begin(), sorted.end(), o2.begin() + b0);
    }
    std::vector<SBlk> sb;
    for (int pass = 0; pass < 2; ++pass) {
        for (int vz = 0; vz < L.n; ++vz)
            for (int c = 0; c < (int)L.c1.size(); ++c) {
                const auto& b = L.c1[c].box;
                if (pass == 0 && !L.c1[c].active) continue;
                if (vz < b.lo[2] || vz >= b.lo[2] + b.num[2] || b.num[0] == 0 || b.num[1] == 0) continue;
                const long long q0 = S.qs_base[c] + (long long)vz * NY * NX;
                const int t1 = (b.lo[1] + b.num[1]) * NX;
                for (int t0 = b.lo[1] * NX; t0 < t1; t0 += SBLOCK)
                    sb.push_back(SBlk{q0, c, vz, t0, std::min(SBLOCK, t1 - t0)});
            }
        if (pass == 0) ctx->nsblks_act = (int)sb.size();
    }
    ctx->nsblks_all = (int)sb.size() - ctx->nsblks_act;
    int rc;
    if ((rc = upload(ctx, &ctx->soff2, o2)) || (rc = upload(ctx, &ctx->sblks, sb)) || (rc = upload_real(ctx, &ctx->qsd, S.qsym)))
        return rc;
    ctx->sg = SymGeo{NX, ctx->pg.H, ctx->pg.NP};
    ctx->use_sym = true;
    // k_qapply_t: every run it copies (aligned down to 16 bytes, SL entries) must lie inside qsym:
    // checked here for every block and slot, else the kernel is not used
    ctx->qt_ok = true;
    {
        const long long al = 16 / (ctx->precision == YGM_FP64 ? 8 : 4);
        const long long SL = ctx->precision == YGM_FP64 ? QtCfg<double>::SL : QtCfg<float>::SL;
        const long long size = (long long)S.qsym.size();
        for (const SBlk& bk : sb) {
            for (int sidx = S.st_begin[bk.cls]; sidx < S.st_begin[bk.cls + 1] && ctx->qt_ok; ++sidx) {
                const long long st = bk.q0 + bk.t0 + o2[sidx].x, lo = st - (st % al + al) % al;
                if (lo < 0 || lo + SL > size) ctx->qt_ok = false;
            }
            if (!ctx->qt_ok) break;
        }
    }
    if (ctx->qt_ok) {
        if ((rc = alloc_dev_err(ctx))) return rc;
        if ((rc = qt_configure(ctx, 0, nullptr))) return rc;
    }
    return 0;
}

// Tables of k_curlT_e_tc: the union U of the merged C^T M2 terms, the dense weights W (curl-carrying
// classes x |U|), the shared-memory layout and the grid.  Requires R in {32, 64, 128}.
static int setup_tc(ygm_ctx* ctx, const std::vector<std::pair<ygm::Nbr, double>>& all, const std::vector<int>& pbeg) {
    const ygm::Lattice& L = ctx->S.L;
    const int R = ctx->n_rhs;
    if (R != 32 && R != 64 && R != 128)
        return fail(ctx, YGM_EINVAL, "tensor-core precisions need n_rhs = 32, 64 or 128 (128 rows = points x columns)");
    std::map<ygm::Nbr, int> kidx;
    for (const auto& t : all) kidx.emplace(t.first, 0);
    int K = 0;
    std::vector<int4> ut;
    for (auto& kv : kidx) {
        kv.second = K++;
        ut.push_back(make_int4(kv.first.cls, kv.first.d[0], kv.first.d[1], kv.first.d[2]));
    }
    std::vector<int> ac;
    for (size_t c = 0; c < L.c1.size(); ++c)
        if (L.c1[c].active) ac.push_back((int)c);
    const int Ma = (int)ac.size(), Kp = (K + 7) / 8 * 8, Nc = std::max(16, (Ma + 15) / 16 * 16);
    if (Nc > 256) return fail(ctx, YGM_EINVAL, "tensor-core C^T M2: more than 256 curl-carrying classes");
    while ((int)ut.size() < Kp) ut.push_back(make_int4(-1, 0, 0, 0));
    std::vector<float> w((size_t)Nc * Kp, 0.f);
    for (int j = 0; j < Ma; ++j)
        for (int t = pbeg[ac[j]]; t < pbeg[ac[j] + 1]; ++t) w[(size_t)j * Kp + kidx[all[t].first]] = (float)all[t].second;
    TcGeo& G = ctx->tcg;
    G.n = L.n;
    G.rshift = ctx->rshift;
    G.P = 128 / R;
    G.nbatch = (int)(((long long)L.n * L.n * L.n + G.P - 1) / G.P);
    G.Kp = Kp;
    G.Nc = Nc;
    G.Ma = Ma;
    G.sboA = Kp / 4 * 128 + 16;
    G.sboB = Kp / 4 * 128 + 16;
    auto al = [](size_t v) { return (int)((v + 1023) / 1024 * 1024); };
    const int aBytes = al((size_t)16 * G.sboA), bBytes = al((size_t)(Nc / 8) * G.sboB);
    const bool three = ctx->tc_passes == 3;
    G.offAlo = aBytes;
    G.offBhi = G.offAlo + (three ? aBytes : 0);
    G.offBlo = G.offBhi + bBytes;
    G.offIdx = G.offBlo + (three ? bBytes : 0);
    G.offBar = G.offIdx + (int)((size_t)G.P * Kp * 4 + 15) / 16 * 16;
    G.tmem_cols = 32;
    while (G.tmem_cols < Nc) G.tmem_cols *= 2;
    ctx->tc_smem = (size_t)G.offBar + 16 + 1024;   // + slack to align the base to 1024 bytes
    if (ctx->tc_smem > 227 * 1024)
        return fail(ctx, YGM_EINVAL, "tensor-core C^T M2 tables exceed shared memory (order 3 is not supported)");
    int rc;
    if ((rc = upload(ctx, &ctx->uterm, ut)) || (rc = upload(ctx, &ctx->acls, ac)) || (rc = upload(ctx, &ctx->wt, w))) return rc;
    if ((rc = alloc_dev_err(ctx))) return rc;
    if (three)
        CK(cudaFuncSetAttribute(k_curlT_e_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->tc_smem));
    else
        CK(cudaFuncSetAttribute(k_curlT_e_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->tc_smem));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int per_sm = std::max(1, (int)((227 * 1024) / ctx->tc_smem));
    ctx->tc_grid = std::min(G.nbatch, nsm * std::min(per_sm, 2));
    return 0;
}

static int setup_device(ygm_ctx* ctx) {
    ygm::Setup& S = ctx->S;
    ygm::Lattice& L = S.L;
    const int k = L.k;
    // padded copies of e (and, for one column, of x and b): halo H = the widest Q1 stencil
    // offset, at least 1 so the curl stencils (offsets within +-1 per axis) fit as well
    int H = 1;
    for (const auto& st : S.st_slots)
        for (int a = 0; a < 3; ++a) H = std::max(H, std::abs((int)st.d[a]));
    const int NP = L.n + 2 * H + 1;
    const long long np3 = (long long)NP * NP * NP;
    if (np3 * (long long)std::max(L.c1.size(), L.c2.size()) * ctx->n_rhs > (long long)INT32_MAX)
        return fail(ctx, YGM_EINVAL, "mesh x n_rhs too large for 32-bit indices of the padded state copies");
    ctx->pg = PadGeo{H, NP};
    ctx->n1pad = np3 * (long long)L.c1.size();
    // classes
    std::vector<DCls> c1(L.c1.size()), c2(L.c2.size());
    std::vector<DInc> inc;
    for (size_t c = 0; c < L.c1.size(); ++c) {
        DCls& D = c1[c];
        for (int a = 0; a < 3; ++a) {
            D.lo[a] = L.c1[c].box.lo[a];
            D.num[a] = L.c1[c].box.num[a];
        }
        D.off = L.c1[c].box.offset;
        D.size = L.c1[c].box.size;
        D.qoff = S.qoff[c];
        D.st_begin = S.st_begin[c];
        D.st_end = S.st_begin[c + 1];
        D.inc_begin = (int)inc.size();
        for (auto& I : L.inc1[c]) inc.push_back(DInc{{I.dcube[0], I.dcube[1], I.dcube[2]}, I.shape, I.loc});
        D.inc_end = (int)inc.size();
        D.pbase = (int)(c * np3);
        D.nup = S.n_upper.empty() ? 0 : S.n_upper[c];
    }
    std::vector<DSlot> slots(S.st_slots.size());
    for (size_t s = 0; s < slots.size(); ++s)
        slots[s] = DSlot{S.st_slots[s].cls, S.st_slots[s].slot, {S.st_slots[s].d[0], S.st_slots[s].d[1], S.st_slots[s].d[2]},
                         S.st_slots[s].upper};
    // integer curl rows of the active 2-form classes (built from the local block of a tet shape
    // that contains the entity: the anchor offsets are relative to the 2-form's own anchor)
    std::vector<DTerm> terms;
    const int n1 = L.n1;
    for (size_t c = 0; c < L.c2.size(); ++c) {
        DCls& D = c2[c];
        for (int a = 0; a < 3; ++a) {
            D.lo[a] = L.c2[c].box.lo[a];
            D.num[a] = L.c2[c].box.num[a];
        }
        D.off = L.c2[c].box.offset;
        D.size = L.c2[c].box.size;
        D.qoff = 0;
        D.inc_begin = D.inc_end = 0;
        D.pbase = (int)(c * np3);
        D.nup = 0;
        D.st_begin = (int)terms.size();
        if (L.c2[c].active) {
            // find a tet shape and local index carrying this class
            bool found = false;
            for (int s = 0; s < 6 && !found; ++s)
                for (int ra = 0; ra < L.n2a && !found; ++ra) {
                    const auto& L2 = L.loc2[s][L.act2[ra]];
                    if (L2.cls != (int)c) continue;
                    for (int j = 0; j < n1; ++j) {
                        int v = S.Cloc[(size_t)ra * n1 + j];
                        if (!v) continue;
                        const auto& L1 = L.loc1[s][j];
                        terms.push_back(DTerm{L1.cls, {L1.off[0] - L2.off[0], L1.off[1] - L2.off[1], L1.off[2] - L2.off[2]}, v});
                    }
                    found = true;
                }
            if (!found) return fail(ctx, YGM_EINVAL, "internal: active 2-form class without a tet");
        }
        D.st_end = (int)terms.size();
    }
    std::vector<DLoc2> loc2;
    for (int s = 0; s < 6; ++s)
        for (int ra = 0; ra < L.n2a; ++ra) {
            const auto& L2 = L.loc2[s][L.act2[ra]];
            loc2.push_back(DLoc2{L2.cls, {L2.off[0], L2.off[1], L2.off[2]}});
        }
    int rc;
    if ((rc = upload(ctx, &ctx->c1, c1)) || (rc = upload(ctx, &ctx->c2, c2)) || (rc = upload(ctx, &ctx->slots, slots)) ||
        (rc = upload(ctx, &ctx->terms, terms)) || (rc = upload(ctx, &ctx->inc, inc)) || (rc = upload(ctx, &ctx->loc2, loc2)))
        return rc;
    if (ctx->n_rhs == 1) {
        // the same curl rows as offsets in the padded geometry (k_curl_b_s)
        std::vector<CTermL> ct(terms.size());
        for (size_t i = 0; i < terms.size(); ++i)
            for (int a = 0; a < 3; ++a)
                if (std::abs(terms[i].d[a]) > H) return fail(ctx, YGM_EINVAL, "internal: curl term beyond the padded halo");
        for (size_t i = 0; i < terms.size(); ++i)
            ct[i] = CTermL{(int)(terms[i].cls * np3 + ((long long)terms[i].d[2] * NP + terms[i].d[1]) * NP + terms[i].d[0]),
                           terms[i].sign};
        if ((rc = upload(ctx, &ctx->cterms, ct))) return rc;
    }
    // rows
    std::vector<DRow> rE = make_rows(L.c1, L.n, true);
    ctx->nrowsE = (int)rE.size();
    if ((rc = upload(ctx, &ctx->rowsE, rE))) return rc;
    // operators
    if ((rc = upload_real(ctx, &ctx->q, S.qvals)) || (rc = upload_real(ctx, &ctx->W, S.Wloc))) return rc;
    std::vector<double> M2a(S.M2aloc);
    if ((rc = upload(ctx, &ctx->M2a, M2a))) return rc;
    bool mu_one = true;
    for (double m : S.mu) mu_one &= (m == 1.0);
    if (!mu_one) {
        std::vector<double> im(S.mu.size());
        for (size_t t = 0; t < im.size(); ++t) im[t] = 1.0 / S.mu[t];
        if ((rc = upload_real(ctx, &ctx->inv_mu, im))) return rc;
    }
    // state
    const size_t R = ctx->n_rhs;
    CK(cudaMalloc(&ctx->e, L.N1 * R * ctx->rs));
    CK(cudaMalloc(&ctx->x, L.N1 * R * ctx->rs));
    CK(cudaMalloc(&ctx->b[0], L.N2 * R * ctx->rs));
    CK(cudaMalloc(&ctx->b[1], L.N2 * R * ctx->rs));
    CK(cudaMalloc(&ctx->bscr, L.N2 * R * ctx->rs));
    CK(cudaMemsetAsync(ctx->e, 0, L.N1 * R * ctx->rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->x, 0, L.N1 * R * ctx->rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[0], 0, L.N2 * R * ctx->rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[1], 0, L.N2 * R * ctx->rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->bscr, 0, L.N2 * R * ctx->rs, ctx->stream));
    ctx->npart = 4 * 152;
    CK(cudaMalloc((void**)&ctx->part, 2 * (size_t)ctx->npart * ctx->n_rhs * sizeof(double2)));
    ctx->hist_cap = 1 << 16;   // records of R values
    CK(cudaMalloc((void**)&ctx->hist, (size_t)ctx->hist_cap * ctx->n_rhs * sizeof(double)));
    ctx->tb = Tables{ctx->c1, ctx->c2, ctx->slots, ctx->terms, ctx->inc, ctx->loc2, L.n, L.n1, L.n2a};
    (void)k;
    // flattened Q1 slot descriptors
    std::vector<QSlot> qs(S.st_slots.size());
    for (size_t c = 0; c < L.c1.size(); ++c)
        for (int sidx = S.st_begin[c]; sidx < S.st_begin[c + 1]; ++sidx) {
            const auto& st = S.st_slots[sidx];
            const auto& D = L.c1[st.cls].box;
            QSlot& Q = qs[sidx];
            Q.ux0 = st.d[0] - D.lo[0];
            Q.uy0 = st.d[1] - D.lo[1];
            Q.uz0 = st.d[2] - D.lo[2];
            Q.nx = D.num[0];
            Q.ny = D.num[1];
            Q.nz = D.num[2];
            Q.ebase = D.offset;
            Q.qbase = st.upper ? S.qoff[c] + (int64_t)st.slot * L.c1[c].box.size : S.qoff[st.cls] + (int64_t)st.slot * D.size;
            Q.upper = st.upper;
            Q.pad = 0;
        }
    if ((rc = upload(ctx, &ctx->qslots, qs))) return rc;
    std::vector<QBlock> qb;
    for (int vz = 0; vz < L.n; ++vz)
        for (int c = 0; c < (int)L.c1.size(); ++c) {
            const auto& b = L.c1[c].box;
            if (vz < b.lo[2] || vz >= b.lo[2] + b.num[2] || b.num[0] == 0 || b.num[1] == 0) continue;
            qb.push_back(QBlock{c, vz});
        }
    ctx->nqblocks = (int)qb.size();
    // k_qapply_p: slot offsets in the padded layout, row blocks, full-row Q1, padded e
    {
        std::vector<int> so(S.st_slots.size());
        for (size_t c = 0; c < L.c1.size(); ++c)
            for (int sidx = S.st_begin[c]; sidx < S.st_begin[c + 1]; ++sidx) {
                const auto& st = S.st_slots[sidx];
                so[sidx] = (int)((((long long)st.cls - (long long)c) * np3 + ((long long)st.d[2] * NP + st.d[1]) * NP + st.d[0])
                                 << ctx->rshift);
            }
        // rows of the curl-carrying classes first: x of a gradient 1-form (a zero column of C) is
        // needed only by the energy, so the steps without an energy read-out skip those rows
        std::vector<PBlk> pb;
        std::vector<int2> planes;
        for (int pass = 0; pass < 2; ++pass) {
            for (int vz = 0; vz < L.n; ++vz)
            for (int c = 0; c < (int)L.c1.size(); ++c) {
                const auto& b = L.c1[c].box;
                if (L.c1[c].active != (pass == 0)) continue;
                if (vz < b.lo[2] || vz >= b.lo[2] + b.num[2] || b.num[0] == 0 || b.num[1] == 0) continue;
                planes.push_back(make_int2(c, vz));
                const int plane = b.num[0] * b.num[1], rz = vz - b.lo[2];
                const long long qplane = S.qf_plane[c];
                const int pz0 = (int)(c * np3) + ((vz + H) * NP + b.lo[1] + H) * NP + b.lo[0] + H;
                const int rows_per = PBLOCK >> ctx->rshift;   // a row owns R threads
                for (int i0 = 0; i0 < plane; i0 += rows_per)
                    pb.push_back(PBlk{i0, std::min(rows_per, plane - i0), b.num[0], pz0, S.st_begin[c],
                                      S.st_begin[c + 1] - S.st_begin[c], (long long)S.qf_off[c] + rz * qplane + i0,
                                      (long long)b.num[2] * qplane, (long long)b.offset + (long long)rz * plane + i0});
            }
            if (pass == 0) ctx->npblks_act = (int)pb.size();
        }
        ctx->npblks = (int)pb.size();
        ctx->nplanes = (int)planes.size();
        if ((rc = upload(ctx, &ctx->soff, so)) || (rc = upload(ctx, &ctx->pblks, pb)) || (rc = upload(ctx, &ctx->planes, planes)))
            return rc;
        for (size_t c = 0; c < L.c1.size(); ++c) ctx->max_ns = std::max(ctx->max_ns, S.st_begin[c + 1] - S.st_begin[c]);
        if ((rc = setup_sym(ctx, so))) return rc;
        // full-row Q1 only where k_qapply_p reads it (R > 1, or offsets beyond 32 bits)
        if (!ctx->use_sym && (rc = upload_real(ctx, &ctx->qf, S.qfull))) return rc;
        // roofline counts of the two launch kinds
        std::vector<char> act(L.N1, 0);
        for (size_t c = 0; c < L.c1.size(); ++c) {
            const auto& b = L.c1[c].box;
            const int64_t stored = (int64_t)(S.st_begin[c + 1] - S.st_begin[c]) * S.qf_plane[c] * b.num[2];
            for (int a = 0; a < 2; ++a)
                if (a == 1 || L.c1[c].active) {
                    ctx->qc_rows[a] += b.size;
                    ctx->qc_stored[a] += stored;
                }
            if (L.c1[c].active) std::fill(act.begin() + b.offset, act.begin() + b.offset + b.size, 1);
        }
        for (int a = 0; a < 2; ++a) {
            int64_t ent = 0, both = 0;   // entries of the computed rows; off-diagonal ones between two such rows
            for (int64_t i = 0; i < L.N1; ++i) {
                if (a == 0 && !act[i]) continue;
                for (int64_t p = S.Q1.ptr[i]; p < S.Q1.ptr[i + 1]; ++p) {
                    ++ent;
                    const int64_t j = S.Q1.col[p];
                    if (j != i && (a == 1 || act[j])) ++both;
                }
            }
            ctx->qc_unique[a] = ent - both / 2;
        }
        CK(cudaMalloc(&ctx->ep, (size_t)ctx->n1pad * ctx->n_rhs * ctx->rs));
        CK(cudaMemsetAsync(ctx->ep, 0, (size_t)ctx->n1pad * ctx->n_rhs * ctx->rs, ctx->stream));
    }
    // k_qapply_b: one warp per TY y-rows of the class box, at most 8 warps per block
    ctx->qthreads = 32 * std::max(1, std::min(WARPS_PER_BLOCK, (L.n + TY - 1) / TY));
    if ((rc = upload(ctx, &ctx->qblocks, qb))) return rc;
    for (size_t c = 0; c < L.c1.size(); ++c) ctx->max_slots = std::max(ctx->max_slots, S.st_begin[c + 1] - S.st_begin[c]);
    std::vector<QBlock> eb, bb;
    for (int vz = 0; vz < L.n; ++vz) {
        for (int c = 0; c < (int)L.c1.size(); ++c) {
            const auto& b = L.c1[c].box;
            if (!L.c1[c].active || vz < b.lo[2] || vz >= b.lo[2] + b.num[2] || b.num[0] == 0 || b.num[1] == 0) continue;
            eb.push_back(QBlock{c, vz});
        }
        for (int c = 0; c < (int)L.c2.size(); ++c) {
            const auto& b = L.c2[c].box;
            if (!L.c2[c].active || vz < b.lo[2] || vz >= b.lo[2] + b.num[2] || b.num[0] == 0 || b.num[1] == 0) continue;
            bb.push_back(QBlock{c, vz});
        }
    }
    ctx->neblocks = (int)eb.size();
    ctx->nbblocks = (int)bb.size();
    if ((rc = upload(ctx, &ctx->eblocks, eb)) || (rc = upload(ctx, &ctx->bblocks, bb))) return rc;
    // merged C^T M2 stencil when mu is uniform
    double mu0 = S.mu.empty() ? 1.0 : S.mu[0];
    bool mu_uniform = true;
    for (double m : S.mu) mu_uniform &= (m == mu0);
    if (mu_uniform) {
        std::vector<int> pbeg(L.c1.size() + 1, 0);
        std::vector<std::pair<ygm::Nbr, double>> all;
        std::vector<std::vector<std::pair<ygm::Nbr, double>>> per(L.c1.size());
        for (size_t c = 0; c < L.c1.size(); ++c) {
            if (!L.c1[c].active) continue;
            std::map<ygm::Nbr, double> acc;
            for (auto& I : L.inc1[c])
                for (int ra = 0; ra < L.n2a; ++ra) {
                    const auto& L2 = L.loc2[I.shape][L.act2[ra]];
                    ygm::Nbr nb{L2.cls, {I.dcube[0] + L2.off[0], I.dcube[1] + L2.off[1], I.dcube[2] + L2.off[2]}};
                    acc[nb] += S.Wloc[(size_t)I.loc * L.n2a + ra] / mu0;
                }
            for (auto& kv : acc) per[c].push_back(kv);
        }
        for (size_t c = 0; c < L.c1.size(); ++c) {
            pbeg[c] = (int)all.size();
            all.insert(all.end(), per[c].begin(), per[c].end());
        }
        pbeg[L.c1.size()] = (int)all.size();
        auto fill = [&](auto* dummy) {
            using R = std::remove_pointer_t<decltype(dummy)>;
            std::vector<PTerm<R>> pt(all.size());
            for (size_t i = 0; i < all.size(); ++i) {
                const auto& nb = all[i].first;
                const auto& D = L.c2[nb.cls].box;
                pt[i] = PTerm<R>{nb.d[0] - D.lo[0], nb.d[1] - D.lo[1], nb.d[2] - D.lo[2], D.num[0], D.num[1], D.num[2],
                                 (long long)D.offset, (R)all[i].second};
            }
            PTerm<R>* d = nullptr;
            int r2 = upload(ctx, &d, pt);
            ctx->pterms = d;
            return r2;
        };
        if (ctx->precision == YGM_FP64) {
            if ((rc = fill((double*)nullptr))) return rc;
        } else {
            if ((rc = fill((float*)nullptr))) return rc;
        }
        if ((rc = upload(ctx, &ctx->pbeg, pbeg))) return rc;
        for (size_t c = 0; c < L.c1.size(); ++c) ctx->max_terms = std::max(ctx->max_terms, pbeg[c + 1] - pbeg[c]);
        if (ctx->tc_passes && (rc = setup_tc(ctx, all, pbeg))) return rc;
        if (ctx->n_rhs == 1) {
            // the same weights as offsets into the padded b (k_curlT_e_s)
            auto wfill = [&](auto* dummy) {
                using R = std::remove_pointer_t<decltype(dummy)>;
                std::vector<WTermL<R>> wt(all.size());
                for (size_t i = 0; i < all.size(); ++i) {
                    const auto& nb = all[i].first;
                    for (int a = 0; a < 3; ++a)
                        if (std::abs(nb.d[a]) > H) return fail(ctx, YGM_EINVAL, "internal: C^T M2 term beyond the padded halo");
                    wt[i] = WTermL<R>{(int)(nb.cls * np3 + ((long long)nb.d[2] * NP + nb.d[1]) * NP + nb.d[0]), (R)all[i].second};
                }
                WTermL<R>* d = nullptr;
                int r2 = upload(ctx, &d, wt);
                ctx->wterms = d;
                return r2;
            };
            if ((rc = ctx->precision == YGM_FP64 ? wfill((double*)nullptr) : wfill((float*)nullptr))) return rc;
        }
    }
    if (ctx->tc_passes && !ctx->wt)
        return fail(ctx, YGM_EINVAL, "tensor-core precisions need a uniform permeability (the merged C^T M2 stencil)");
    // lattice block lists of the padded curl kernels (one column, with k_qapply_s)
    if (ctx->use_sym) {
        const int NX = ctx->sg.NX;
        auto blocks_of = [&](const std::vector<ygm::DofClass>& cls) {
            std::vector<SBlk> out;
            for (int vz = 0; vz < L.n; ++vz)
                for (int c = 0; c < (int)cls.size(); ++c) {
                    const auto& b = cls[c].box;
                    if (!cls[c].active) continue;
                    if (vz < b.lo[2] || vz >= b.lo[2] + b.num[2] || b.num[0] == 0 || b.num[1] == 0) continue;
                    const int t1 = (b.lo[1] + b.num[1]) * NX;
                    for (int t0 = b.lo[1] * NX; t0 < t1; t0 += SBLOCK)
                        out.push_back(SBlk{0, c, vz, t0, std::min(SBLOCK, t1 - t0)});
                }
            return out;
        };
        std::vector<SBlk> lb = blocks_of(L.c2), le = blocks_of(L.c1);
        ctx->nlb = (int)lb.size();
        ctx->nle = (int)le.size();
        if ((rc = upload(ctx, &ctx->lblks_b, lb)) || (rc = upload(ctx, &ctx->lblks_e, le))) return rc;
        ctx->h_lblks_e = le;
        const size_t n2pad = (size_t)np3 * L.c2.size();
        CK(cudaMalloc(&ctx->xp, (size_t)ctx->n1pad * ctx->rs));
        CK(cudaMalloc(&ctx->bp, n2pad * ctx->rs));
        CK(cudaMemsetAsync(ctx->xp, 0, (size_t)ctx->n1pad * ctx->rs, ctx->stream));
        CK(cudaMemsetAsync(ctx->bp, 0, n2pad * ctx->rs, ctx->stream));
    }
    if (ctx->use_sym) {
        // fused energy of one column: e_i x_i partials of the Q1 apply, the tet-sum counter, M2a
        CK(cudaMalloc((void**)&ctx->qpart, (size_t)std::max(1, ctx->nsblks_all) * sizeof(double2)));
        CK(cudaMalloc((void**)&ctx->ticket, sizeof(unsigned)));
        CK(cudaMemsetAsync(ctx->ticket, 0, sizeof(unsigned), ctx->stream));
        if ((rc = upload_real(ctx, &ctx->M2af, S.M2aloc))) return rc;
    }
    for (int i = 0; i < 2; ++i) CK(cudaEventCreateWithFlags(&ctx->damp_ev[i], cudaEventDisableTiming));
    // dynamic shared memory of the block kernels (slot / term tables of one class); above 48 KB
    // the kernels must opt in, up to the 227 KB per-CTA limit of sm_103a
    const size_t smem_q = (size_t)ctx->max_slots * (2 * sizeof(long long) + 8 * sizeof(int));
    const size_t smem_e = (size_t)ctx->max_terms * sizeof(long long) + (size_t)(ctx->max_terms + 1) * ctx->rs +
                          (size_t)ctx->max_terms * 6 * sizeof(int);
    if (smem_q > 227 * 1024 || smem_e > 227 * 1024 || (size_t)ctx->max_ns * sizeof(int) > 48 * 1024)
        return fail(ctx, YGM_EINVAL, "stencil too wide for shared memory");
    // raise-only: the limit is process-wide per kernel, shared by every context (a smaller value
    // set by one context would make another context's launches invalid)
    {
        std::lock_guard<std::mutex> lk(g_smem_mutex);
        size_t& lim_q = smem_limit(g_smem_q, ctx->device, ctx->precision);
        size_t& lim_e = smem_limit(g_smem_e, ctx->device, ctx->precision);
        if (smem_q > lim_q) {
            if (smem_q > 48 * 1024) {
                if (ctx->precision == YGM_FP64)
                    CK(cudaFuncSetAttribute(k_qapply_b<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_q));
                else
                    CK(cudaFuncSetAttribute(k_qapply_b<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_q));
            }
            lim_q = smem_q;
        }
        if (smem_e > lim_e) {
            if (smem_e > 48 * 1024) {
                if (ctx->precision == YGM_FP64)
                    CK(cudaFuncSetAttribute(k_curlT_e_b<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e));
                else
                    CK(cudaFuncSetAttribute(k_curlT_e_b<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e));
            }
            lim_e = smem_e;
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

// ------------------------------------------------------------------ launch helpers
// One kernel launch on the context stream; with ctx->pdl the launch carries programmatic stream
// serialization, so the kernel's blocks may start while the previous kernel of the stream is
// finishing (the kernel waits for it with pdl_wait before touching its output).
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(const ygm_ctx* ctx, void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = ctx->pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
// x = Q1 e of the context state, read from the padded copy of e; all_rows = false computes only
// the rows of the curl-carrying 1-forms (all that C x needs).  On the upper-triangle path an
// all-rows apply also leaves the per-block e_i x_i partials of W_n in ctx->qpart.
static int launch_qapply(ygm_ctx* ctx, void* x, bool all_rows) {
    if (ctx->use_sym) {
        const int nb = all_rows ? ctx->nsblks_all : ctx->nsblks_act;
        if (!nb) return 0;
        const SBlk* blks = ctx->sblks + (all_rows ? ctx->nsblks_act : 0);
        time_begin(ctx, KQ);
        const size_t smem = (size_t)(ctx->max_ns + 8) * sizeof(int2);
        if (ctx->qt_ok && ctx->qt_mode == 2) {
            if (ctx->precision == YGM_FP64) {
                auto k = all_rows ? k_qapply_t<double, true> : k_qapply_t<double, false>;
                k<<<nb, QT_THREADS, ctx->qt_smem, ctx->stream>>>(blks, ctx->c1, ctx->soff2, ctx->sg, (const double*)ctx->qsd,
                                                              (const double*)ctx->ep, (double*)x, (double*)ctx->xp, ctx->qpart,
                                                              ctx->qt_nst, ctx->dev_err);
            } else {
                auto k = all_rows ? k_qapply_t<float, true> : k_qapply_t<float, false>;
                k<<<nb, QT_THREADS, ctx->qt_smem, ctx->stream>>>(blks, ctx->c1, ctx->soff2, ctx->sg, (const float*)ctx->qsd,
                                                              (const float*)ctx->ep, (float*)x, (float*)ctx->xp, ctx->qpart,
                                                              ctx->qt_nst, ctx->dev_err);
            }
        } else if (ctx->precision == YGM_FP64) {
            auto k = all_rows ? k_qapply_s<double, true> : k_qapply_s<double, false>;
            CK(launch_k(ctx, k, nb, SBLOCK, smem, blks, ctx->c1, ctx->soff2, ctx->sg, (const double*)ctx->qsd,
                        (const double*)ctx->ep, (double*)x, (double*)ctx->xp, ctx->qpart));
        } else {
            auto k = all_rows ? k_qapply_s<float, true> : k_qapply_s<float, false>;
            CK(launch_k(ctx, k, nb, SBLOCK, smem, blks, ctx->c1, ctx->soff2, ctx->sg, (const float*)ctx->qsd,
                        (const float*)ctx->ep, (float*)x, (float*)ctx->xp, ctx->qpart));
        }
        time_end(ctx);
        ctx->launches++;
        return 0;
    }
    const int nb = all_rows ? ctx->npblks : ctx->npblks_act;
    if (!nb) return 0;
    time_begin(ctx, KQ);
    const size_t smem = (size_t)ctx->max_ns * sizeof(int);
    if (ctx->precision == YGM_FP64)
        k_qapply_p<double><<<nb, PBLOCK, smem, ctx->stream>>>(ctx->pblks, ctx->soff, ctx->pg.NP, ctx->rshift, (const double*)ctx->qf,
                                                              (const double*)ctx->ep, (double*)x);
    else
        k_qapply_p<float><<<nb, PBLOCK, smem, ctx->stream>>>(ctx->pblks, ctx->soff, ctx->pg.NP, ctx->rshift, (const float*)ctx->qf,
                                                             (const float*)ctx->ep, (float*)x);
    time_end(ctx);
    ctx->launches++;
    return 0;
}
// R > 1 plane kernels: blockIdx.x picks the (class, z-plane), blockIdx.y a slice of its n^2 * R items
static dim3 plane_grid(const ygm_ctx* ctx, int nblocks) {
    const long long items = (long long)ctx->S.L.n * ctx->S.L.n * ctx->n_rhs;
    return dim3((unsigned)nblocks, (unsigned)std::min<long long>(65535, (items + BLOCK - 1) / BLOCK));
}
static int launch_curl_b(ygm_ctx* ctx, const void* x, const void* bin, void* bout, double ctau) {
    if (!ctx->nbblocks) return 0;
    time_begin(ctx, KB);
    if (ctx->use_sym && ctx->nlb) {      // x was written to its padded copy by k_qapply_s
        if (ctx->precision == YGM_FP64)
            CK(launch_k(ctx, k_curl_b_s<double>, ctx->nlb, SBLOCK, 0, ctx->lblks_b, ctx->c2, ctx->cterms, ctx->pg, ctx->sg.NX,
                        (const double*)ctx->xp, (const double*)bin, (double*)bout, (double*)ctx->bp, split_tau<double>(ctau)));
        else
            CK(launch_k(ctx, k_curl_b_s<float>, ctx->nlb, SBLOCK, 0, ctx->lblks_b, ctx->c2, ctx->cterms, ctx->pg, ctx->sg.NX,
                        (const float*)ctx->xp, (const float*)bin, (float*)bout, (float*)ctx->bp, split_tau<float>(ctau)));
    } else if (ctx->rshift) {
        if (ctx->precision == YGM_FP64)
            k_curl_b_r<double><<<ctx->nbblocks, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->c2, ctx->terms, ctx->bblocks, ctx->rshift,
                                                                         (const double*)x, (const double*)bin, (double*)bout, ctau);
        else
            k_curl_b_r<float><<<ctx->nbblocks, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->c2, ctx->terms, ctx->bblocks, ctx->rshift,
                                                                        (const float*)x, (const float*)bin, (float*)bout,
                                                                        (float)ctau);
    } else if (ctx->precision == YGM_FP64)
        k_curl_b_b<double><<<ctx->nbblocks, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->c2, ctx->terms, ctx->bblocks,
                                                                     (const double*)x, (const double*)bin, (double*)bout, ctau);
    else
        k_curl_b_b<float><<<ctx->nbblocks, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->c2, ctx->terms, ctx->bblocks,
                                                                    (const float*)x, (const float*)bin, (float*)bout,
                                                                    (float)ctau);
    time_end(ctx);
    ctx->launches++;
    return 0;
}
static int launch_source(ygm_ctx* ctx, const double* amp_dev);
// e += ctau C^T M2 b, then the dipole currents of this step when amp_dev != NULL (amp_dev =
// this step's dt s(t_{n+1/2}) per source).  The one-column lattice path does both in one pass;
// the other paths follow the e update with k_source.
static int launch_curlT_e(ygm_ctx* ctx, const void* b, void* e, double ctau, const double* amp_dev) {
    time_begin(ctx, KE);
    if (ctx->use_sym && ctx->nlb && ctx->wterms && ctx->nle) {   // b was written to its padded copy by k_curl_b_s
        const size_t smem = (size_t)ctx->max_terms * (ctx->precision == YGM_FP64 ? sizeof(WTermL<double>) : sizeof(WTermL<float>));
        const bool src = amp_dev && ctx->nsrc && ctx->lblks_es;
        const SBlk* blks = src ? ctx->lblks_es : ctx->lblks_e;
        const int nb = src ? ctx->nle_src : ctx->nle;
        const double* amp = src ? amp_dev : nullptr;
        if (ctx->precision == YGM_FP64)
            CK(launch_k(ctx, k_curlT_e_s<double>, nb, SBLOCK, smem, blks, ctx->c1, ctx->pbeg, (const WTermL<double>*)ctx->wterms,
                        ctx->pg, ctx->sg.NX, (const double*)ctx->bp, (double*)e, split_tau<double>(ctau), (double*)ctx->ep,
                        ctx->sbeg, (const SrcE<double>*)ctx->sent, amp));
        else
            CK(launch_k(ctx, k_curlT_e_s<float>, nb, SBLOCK, smem, blks, ctx->c1, ctx->pbeg, (const WTermL<float>*)ctx->wterms,
                        ctx->pg, ctx->sg.NX, (const float*)ctx->bp, (float*)e, split_tau<float>(ctau), (float*)ctx->ep,
                        ctx->sbeg, (const SrcE<float>*)ctx->sent, amp));
        time_end(ctx);
        ctx->launches++;
        return 0;
    } else if (ctx->rshift) {
        if (!ctx->neblocks) {
        } else if (ctx->tc_passes && ctx->wt) {
            auto k = ctx->tc_passes == 3 ? k_curlT_e_tc<3> : k_curlT_e_tc<1>;
            const int thr = ctx->tc_passes == 3 ? tc_threads<3>() : tc_threads<1>();
            k<<<ctx->tc_grid, thr, ctx->tc_smem, ctx->stream>>>(ctx->tcg, ctx->uterm, ctx->c1, ctx->c2, ctx->acls, ctx->wt,
                                                               (const float*)b, (float*)e, (float*)ctx->ep, ctx->pg,
                                                               split_tau<float>(ctau), ctx->dev_err);
        } else if (ctx->pterms) {
            const size_t smem = (size_t)ctx->max_terms * (ctx->precision == YGM_FP64 ? sizeof(PTerm<double>) : sizeof(PTerm<float>));
            if (ctx->precision == YGM_FP64)
                k_curlT_e_r<double><<<plane_grid(ctx, ctx->neblocks), BLOCK, smem, ctx->stream>>>(
                    ctx->c1, ctx->pbeg, (const PTerm<double>*)ctx->pterms, ctx->eblocks, ctx->rshift, (const double*)b,
                    (double*)e, ctau, (double*)ctx->ep, ctx->pg);
            else
                k_curlT_e_r<float><<<plane_grid(ctx, ctx->neblocks), BLOCK, smem, ctx->stream>>>(
                    ctx->c1, ctx->pbeg, (const PTerm<float>*)ctx->pterms, ctx->eblocks, ctx->rshift, (const float*)b,
                    (float*)e, (float)ctau, (float*)ctx->ep, ctx->pg);
        } else {
            if (ctx->precision == YGM_FP64)
                k_curlT_e_rt<double><<<plane_grid(ctx, ctx->neblocks), BLOCK, 0, ctx->stream>>>(
                    ctx->tb, ctx->eblocks, ctx->rshift, (const double*)ctx->W, (const double*)b, (const double*)ctx->inv_mu,
                    (double*)e, ctau, (double*)ctx->ep, ctx->pg);
            else
                k_curlT_e_rt<float><<<plane_grid(ctx, ctx->neblocks), BLOCK, 0, ctx->stream>>>(
                    ctx->tb, ctx->eblocks, ctx->rshift, (const float*)ctx->W, (const float*)b, (const float*)ctx->inv_mu,
                    (float*)e, (float)ctau, (float*)ctx->ep, ctx->pg);
        }
    } else if (ctx->pterms) {
        const int mt = ctx->max_terms;
        const size_t smem = (size_t)mt * sizeof(long long) + (size_t)(mt + (mt & 1)) * ctx->rs + (size_t)mt * 6 * sizeof(int);
        if (ctx->neblocks) {
            if (ctx->precision == YGM_FP64)
                k_curlT_e_b<double><<<ctx->neblocks, BLOCK, smem, ctx->stream>>>(
                    ctx->c1, ctx->pbeg, (const PTerm<double>*)ctx->pterms, ctx->eblocks, mt, (const double*)b, (double*)e, ctau,
                    (double*)ctx->ep, ctx->pg);
            else
                k_curlT_e_b<float><<<ctx->neblocks, BLOCK, smem, ctx->stream>>>(
                    ctx->c1, ctx->pbeg, (const PTerm<float>*)ctx->pterms, ctx->eblocks, mt, (const float*)b, (float*)e,
                    (float)ctau, (float*)ctx->ep, ctx->pg);
        }
    } else {
        dim3 g((ctx->nrowsE + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
        if (ctx->precision == YGM_FP64)
            k_curlT_e<double><<<g, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->rowsE, ctx->nrowsE, (const double*)ctx->W,
                                                            (const double*)b, (const double*)ctx->inv_mu, (double*)e, ctau,
                                                            (double*)ctx->ep, ctx->pg);
        else
            k_curlT_e<float><<<g, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->rowsE, ctx->nrowsE, (const float*)ctx->W,
                                                           (const float*)b, (const float*)ctx->inv_mu, (float*)e,
                                                           (float)ctau, (float*)ctx->ep, ctx->pg);
    }
    time_end(ctx);
    ctx->launches++;
    if (amp_dev) return launch_source(ctx, amp_dev);
    return 0;
}
static int launch_source(ygm_ctx* ctx, const double* amp_dev) {
    if (!ctx->nsrc) return 0;
    time_begin(ctx, KS);
    if (ctx->precision == YGM_FP64)
        k_source<double><<<1, 256, 0, ctx->stream>>>(ctx->dsrc, ctx->nsrc, ctx->sdofs, ctx->spdofs, (const double*)ctx->sw,
                                                     amp_dev, (double*)ctx->e, (double*)ctx->ep);
    else
        k_source<float><<<1, 256, 0, ctx->stream>>>(ctx->dsrc, ctx->nsrc, ctx->sdofs, ctx->spdofs, (const float*)ctx->sw,
                                                    amp_dev, (float*)ctx->e, (float*)ctx->ep);
    time_end(ctx);
    ctx->launches++;
    return 0;
}
// refresh the padded copy of e after the compact state was overwritten
static int launch_pad_e(ygm_ctx* ctx) {
    if (!ctx->nplanes) return 0;
    if (ctx->precision == YGM_FP64)
        k_pad_e<double><<<ctx->nplanes, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->planes, ctx->pg, ctx->rshift, (const double*)ctx->e,
                                                                 (double*)ctx->ep);
    else
        k_pad_e<float><<<ctx->nplanes, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->planes, ctx->pg, ctx->rshift, (const float*)ctx->e,
                                                                (float*)ctx->ep);
    ctx->launches++;
    return 0;
}
// out = 1/2 e^T x + 1/2 sum_T bn^T M2 bo / mu_T  (device double)
static int launch_energy(ygm_ctx* ctx, const void* e, const void* x, const void* bn, const void* bo, double* out) {
    const int np = ctx->npart;
    const long long N1 = ctx->S.L.N1;
    time_begin(ctx, KW);
    if (ctx->rshift) {   // out[R]
        const int R = ctx->n_rhs;
        double2* p2 = ctx->part + (size_t)np * R;
        if (ctx->precision == YGM_FP64) {
            k_dot_r<double><<<np, BLOCK, 0, ctx->stream>>>((const double*)e, (const double*)x, N1, ctx->rshift, ctx->part);
            k_tet_quad_r<double><<<np, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->M2a, (const double*)bn, (const double*)bo,
                                                                (const double*)ctx->inv_mu, ctx->rshift, p2);
        } else {
            k_dot_r<float><<<np, BLOCK, 0, ctx->stream>>>((const float*)e, (const float*)x, N1, ctx->rshift, ctx->part);
            k_tet_quad_r<float><<<np, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->M2a, (const float*)bn, (const float*)bo,
                                                               (const float*)ctx->inv_mu, ctx->rshift, p2);
        }
        k_finish_r<<<1, 256, 0, ctx->stream>>>(ctx->part, p2, np, R, out);
        time_end(ctx);
        ctx->launches += 3;
        return 0;
    }
    if (ctx->use_sym && ctx->qpart) {
        // e^T x was summed by the all-rows k_qapply_s that produced x (per-block partials)
        if (ctx->precision == YGM_FP64)
            k_tet_energy<double, double><<<np, BLOCK, 0, ctx->stream>>>(ctx->tb, (const double*)ctx->M2af, (const double*)bn,
                                                                        (const double*)bo, (const double*)ctx->inv_mu, ctx->part,
                                                                        ctx->qpart, ctx->nsblks_all, ctx->ticket, out);
        else
            k_tet_energy<float, float><<<np, BLOCK, 0, ctx->stream>>>(ctx->tb, (const float*)ctx->M2af, (const float*)bn,
                                                                      (const float*)bo, (const float*)ctx->inv_mu, ctx->part,
                                                                      ctx->qpart, ctx->nsblks_all, ctx->ticket, out);
        time_end(ctx);
        ctx->launches++;
        return 0;
    }
    if (ctx->precision == YGM_FP64) {
        k_dot<double><<<np, BLOCK, 0, ctx->stream>>>((const double*)e, (const double*)x, N1, ctx->part);
        k_tet_quad<double><<<np, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->M2a, (const double*)bn, (const double*)bo,
                                                          (const double*)ctx->inv_mu, ctx->part + np);
    } else {
        k_dot<float><<<np, BLOCK, 0, ctx->stream>>>((const float*)e, (const float*)x, N1, ctx->part);
        k_tet_quad<float><<<np, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->M2a, (const float*)bn, (const float*)bo,
                                                         (const float*)ctx->inv_mu, ctx->part + np);
    }
    k_finish<<<1, 1024, 0, ctx->stream>>>(ctx->part, np, ctx->part + np, np, out);
    time_end(ctx);
    ctx->launches += 3;
    return 0;
}

// Device-side failures reported through flags (a tensor-core MMA wait that gave up): checked by
// the calls that synchronise the stream anyway.
static int check_device_flags(ygm_ctx* ctx) {
    if (!ctx->dev_err) return 0;
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h & 1) return fail(ctx, YGM_ETIMEOUT, "a tensor-core MMA completion wait gave up (k_curlT_e_tc); results are invalid");
    if (h & QT_ERR_BIT)
        return fail(ctx, YGM_ETIMEOUT, "a Q1 bulk-copy completion wait gave up (k_qapply_t); results are invalid");
    return 0;
}

// ====================================================================== no-allocation step
// Callers that must not allocate device memory (a process whose device memory is reserved up
// front by another allocator, or code under a real-time budget that rules out cudaMalloc and its
// possible device synchronisation) still need the Q1 e scratch
// vector of a leapfrog step.  It lives in this fixed, file-scope device array instead: every
// GPU that loads the library holds these 16 MiB until the process exits.  Host code must not
// pass the symbol itself to a kernel (on the host it is only a stand-in): its device address
// is obtained once per device with cudaGetSymbolAddress.
constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
static void* g_noalloc_addr[256] = {nullptr};
static std::mutex g_noalloc_mutex;

extern "C" {

const char* ygm_last_error(const ygm_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mutex);
    return g_create_err.c_str();
}

static int finish_create(ygm_ctx* ctx, const ygm_opts& o, ygm_ctx** out);

int ygm_create(const ygm_mesh* mesh, int order, const double* eps, const double* mu, const ygm_opts* opts,
               ygm_ctx** out) {
    auto cerr = [](int code, const std::string& m) {
        std::lock_guard<std::mutex> lk(g_err_mutex);
        g_create_err = m;
        return code;
    };
    if (!out) return cerr(YGM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || mesh->n < 1 || !(mesh->side > 0) || !std::isfinite(mesh->side))
        return cerr(YGM_EINVAL, "mesh: need n >= 1 and finite side > 0");
    if (order < 1 || order > 3) return cerr(YGM_EINVAL, "order must be 1, 2 or 3");
    ygm_opts o{};
    o.precision = YGM_FP64;
    o.n_rhs = 1;
    if (opts) o = *opts;
    if (o.precision < YGM_FP64 || o.precision > YGM_FP32_TC_3XTF32)
        return cerr(YGM_EINVAL, "precision must be YGM_FP64, YGM_FP32, YGM_FP32_TC_TF32 or YGM_FP32_TC_3XTF32");
    if (o.n_rhs < 1 || o.n_rhs > 256 || (o.n_rhs & (o.n_rhs - 1)))
        return cerr(YGM_EINVAL, "n_rhs must be a power of two in [1, 256]");
    if (o.energy_every < 0) return cerr(YGM_EINVAL, "energy_every must be >= 0");
    if (o.q1_pattern < 0 || o.q1_pattern > 3) return cerr(YGM_EINVAL, "unknown q1_pattern");
    const bool host_only = o.device == -1;
    int ndev = 0;
    if (!host_only) {
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return cerr(YGM_ENODEV, "no CUDA device");
        if (o.device < 0 || o.device >= ndev) return cerr(YGM_EINVAL, "device ordinal out of range");
    }
    ygm_ctx* ctx = new (std::nothrow) ygm_ctx();
    if (!ctx) return cerr(YGM_ENOMEM, "host allocation failed");
    int rc = ygm::build_setup(ctx->S, mesh->n, mesh->side, order, eps, mu, o.q1_pattern, o.threads);
    if (rc) {
        std::string m = ctx->S.err;
        delete ctx;
        return cerr(rc == -1 ? YGM_EINVAL : YGM_ENOTSPD, m);
    }
    return finish_create(ctx, o, out);
}

// Second half of context creation: the options, the stream and the device copies of an
// already built host set-up (ctx->S).  Takes ownership of ctx.
static int finish_create(ygm_ctx* ctx, const ygm_opts& o, ygm_ctx** out) {
    // tensor-core precisions keep FP32 state and FP32 SIMT kernels except the C^T M2 contraction
    ctx->tc_passes = o.precision == YGM_FP32_TC_TF32 ? 1 : o.precision == YGM_FP32_TC_3XTF32 ? 3 : 0;
    ctx->precision = o.precision == YGM_FP64 ? YGM_FP64 : YGM_FP32;
    ctx->rs = o.precision == YGM_FP64 ? 8 : 4;
    ctx->n_rhs = o.n_rhs;
    ctx->rshift = 0;
    while ((1 << ctx->rshift) < o.n_rhs) ++ctx->rshift;
    ctx->energy_every = o.energy_every;
    ctx->device = o.device;
    ctx->host_only = o.device == -1;
    if (ctx->host_only) {
        *out = ctx;
        return YGM_OK;
    }
    auto cerr = [&](int code, const std::string& m) {
        std::lock_guard<std::mutex> lk(g_err_mutex);
        g_create_err = m;
        return code;
    };
    if (cudaSetDevice(o.device) != cudaSuccess) {
        delete ctx;
        return cerr(YGM_ECUDA, "cudaSetDevice failed");
    }
    if (o.stream) {
        ctx->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return cerr(YGM_ECUDA, "cudaStreamCreate failed");
        }
        ctx->own_stream = true;
    }
    int rc = setup_device(ctx);
    if (rc) {
        std::string m = ctx->err;
        ygm_destroy(ctx);
        return cerr(rc, m);
    }
    *out = ctx;
    return YGM_OK;
}

int ygm_create_like(const ygm_ctx* src, const ygm_opts* opts, ygm_ctx** out) {
    auto cerr = [](int code, const std::string& m) {
        std::lock_guard<std::mutex> lk(g_err_mutex);
        g_create_err = m;
        return code;
    };
    if (!out) return cerr(YGM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!src) return cerr(YGM_EINVAL, "src is NULL");
    ygm_opts o{};
    o.precision = YGM_FP64;
    o.n_rhs = 1;
    if (opts) o = *opts;
    if (o.precision < YGM_FP64 || o.precision > YGM_FP32_TC_3XTF32)
        return cerr(YGM_EINVAL, "precision must be YGM_FP64, YGM_FP32, YGM_FP32_TC_TF32 or YGM_FP32_TC_3XTF32");
    if (o.n_rhs < 1 || o.n_rhs > 256 || (o.n_rhs & (o.n_rhs - 1)))
        return cerr(YGM_EINVAL, "n_rhs must be a power of two in [1, 256]");
    if (o.energy_every < 0) return cerr(YGM_EINVAL, "energy_every must be >= 0");
    if (o.device != -1) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return cerr(YGM_ENODEV, "no CUDA device");
        if (o.device < 0 || o.device >= ndev) return cerr(YGM_EINVAL, "device ordinal out of range");
    }
    ygm_ctx* ctx = new (std::nothrow) ygm_ctx();
    if (!ctx) return cerr(YGM_ENOMEM, "host allocation failed");
    try {
        ctx->S = src->S;
    } catch (const std::exception& ex) {
        delete ctx;
        return cerr(YGM_ENOMEM, std::string("copying the host set-up failed: ") + ex.what());
    }
    return finish_create(ctx, o, out);
}

int ygm_sizes(const ygm_ctx* ctx, int64_t* n1, int64_t* n2, int64_t* q1_nnz, double* dt_cfl) {
    if (!ctx) return YGM_EINVAL;
    if (n1) *n1 = ctx->S.L.N1;
    if (n2) *n2 = ctx->S.L.N2;
    if (q1_nnz) *q1_nnz = (int64_t)ctx->S.Q1.col.size();
    if (dt_cfl) *dt_cfl = ctx->S.tau_cfl;
    return YGM_OK;
}

int ygm_set_state(ygm_ctx* ctx, const void* e, const void* b, int on_device) {
    if (ctx && ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (!ctx || !e || !b) return fail(ctx, YGM_EINVAL, "NULL argument");
    const size_t ne = ctx->S.L.N1 * ctx->n_rhs * ctx->rs, nb = ctx->S.L.N2 * ctx->n_rhs * ctx->rs;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(ctx->e, e, ne, kind, ctx->stream));
    CK(cudaMemcpyAsync(ctx->b[0], b, nb, kind, ctx->stream));
    CK(cudaMemcpyAsync(ctx->b[1], b, nb, kind, ctx->stream));
    launch_pad_e(ctx);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    ctx->cur = 0;
    ctx->staggered = false;
    ctx->step = ctx->step_base = 0;
    ctx->t_base = 0.0;
    ctx->hist_n = 0;
    return YGM_OK;
}

int ygm_get_state(ygm_ctx* ctx, void* e, void* b, int on_device, int synced) {
    if (ctx && ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (!ctx) return YGM_EINVAL;
    const size_t ne = ctx->S.L.N1 * ctx->n_rhs * ctx->rs, nb = ctx->S.L.N2 * ctx->n_rhs * ctx->rs;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e) CK(cudaMemcpyAsync(e, ctx->e, ne, kind, ctx->stream));
    if (b) {
        const void* src = ctx->b[ctx->cur];
        if (synced && ctx->staggered) {
            CK(cudaMemcpyAsync(ctx->bscr, ctx->b[ctx->cur], nb, cudaMemcpyDeviceToDevice, ctx->stream));
            launch_qapply(ctx, ctx->x, false);
            launch_curl_b(ctx, ctx->x, ctx->b[ctx->cur], ctx->bscr, 0.5 * ctx->split_w[0] * ctx->dt_prev);
            src = ctx->bscr;
        }
        CK(cudaMemcpyAsync(b, src, nb, kind, ctx->stream));
    }
    CK(cudaGetLastError());
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return check_device_flags(ctx);
}

int ygm_project_E(ygm_ctx* ctx, void (*E0)(const double x[3], double out[3], void* user), void* user, int32_t rhs) {
    if (ctx && ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (!ctx || !E0) return fail(ctx, YGM_EINVAL, "NULL argument");
    if (rhs < 0 || rhs >= ctx->n_rhs) return fail(ctx, YGM_EINVAL, "rhs out of range");
    std::vector<double> e0;
    ygm::project_E(ctx->S, E0, user, e0, 1);
    std::vector<double> bz(ctx->S.L.N2, 0.0);
    int rc;
    void* de = nullptr;
    if ((rc = upload_real(ctx, &de, e0))) return rc;
    // column rhs of the [N1][R] state (a strided copy for R > 1); the other columns keep their e
    CK(cudaMemcpy2DAsync((char*)ctx->e + (size_t)rhs * ctx->rs, (size_t)ctx->n_rhs * ctx->rs, de, ctx->rs, ctx->rs,
                         e0.size(), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[0], 0, bz.size() * ctx->n_rhs * ctx->rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[1], 0, bz.size() * ctx->n_rhs * ctx->rs, ctx->stream));
    launch_pad_e(ctx);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(de);
    ctx->cur = 0;
    ctx->staggered = false;
    ctx->step = ctx->step_base = 0;
    ctx->t_base = 0.0;
    ctx->hist_n = 0;
    return YGM_OK;
}

static int set_sources(ygm_ctx* ctx, const ygm_source* src, int32_t n_src) {
    bool same = (int)ctx->src_cache.size() == n_src;
    for (int i = 0; same && i < n_src; ++i) same = std::memcmp(&ctx->src_cache[i], &src[i], sizeof(ygm_source)) == 0;
    if (same) return 0;
    std::vector<DSrc> hs;
    std::vector<long long> dofs;
    std::vector<int> pdofs;
    std::vector<double> w;
    for (int i = 0; i < n_src; ++i) {
        const ygm_source& s = src[i];
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(s.x[a]) || !std::isfinite(s.d[a]) || s.x[a] < 0 || s.x[a] > ctx->S.L.h * ctx->S.L.n)
                return fail(ctx, YGM_EINVAL, "source position outside the cube or not finite");
        if (!(s.sigma > 0) || !std::isfinite(s.amp) || !std::isfinite(s.omega) || !std::isfinite(s.t0))
            return fail(ctx, YGM_EINVAL, "source parameters invalid (sigma must be > 0)");
        if (s.rhs < 0 || s.rhs >= ctx->n_rhs) return fail(ctx, YGM_EINVAL, "source rhs out of range");
        std::vector<int64_t> d;
        std::vector<double> ww;
        if (ygm::dipole_weights(ctx->S, s.x, s.d, d, ww)) return fail(ctx, YGM_EINVAL, "source not located");
        DSrc ds{(int)dofs.size(), 0};
        for (size_t j = 0; j < d.size(); ++j) {
            dofs.push_back(d[j] * ctx->n_rhs + s.rhs);
            w.push_back(ww[j]);
            int cls, v[3];
            ctx->S.L.decode1(d[j], &cls, v);
            const int H = ctx->pg.H, NP = ctx->pg.NP;
            pdofs.push_back((int)((((long long)cls * NP * NP * NP + ((long long)(v[2] + H) * NP + v[1] + H) * NP + v[0] + H)
                                   << ctx->rshift) + s.rhs));
        }
        ds.end = (int)dofs.size();
        hs.push_back(ds);
    }
    // one-column lattice path: the source entries of each k_curlT_e_s block, with extra blocks
    // for curl-free classes (gradient 1-forms) that hold a source DoF
    std::vector<SBlk> comb;
    std::vector<int> sb;
    std::vector<std::pair<int, std::pair<int, std::pair<int, double>>>> ent;   // (block, (tid, (source, w)))
    if (ctx->use_sym && ctx->nle && ctx->n_rhs == 1) {
        comb = ctx->h_lblks_e;
        std::map<std::array<int, 3>, int> blk_of;
        for (size_t i = 0; i < comb.size(); ++i) blk_of[{comb[i].cls, comb[i].vz, comb[i].t0}] = (int)i;
        const int NX = ctx->sg.NX;
        for (int q = 0; q < n_src; ++q)
            for (int j = hs[q].begin; j < hs[q].end; ++j) {
                int cls, v[3];
                ctx->S.L.decode1(dofs[j], &cls, v);
                const auto& bx = ctx->S.L.c1[cls].box;
                const int t = v[1] * NX + v[0], base = bx.lo[1] * NX, t1 = (bx.lo[1] + bx.num[1]) * NX;
                const int t0 = base + (t - base) / SBLOCK * SBLOCK;
                auto it = blk_of.find({cls, v[2], t0});
                int bi;
                if (it == blk_of.end()) {
                    bi = (int)comb.size();
                    comb.push_back(SBlk{0, cls, v[2], t0, std::min(SBLOCK, t1 - t0)});
                    blk_of[{cls, v[2], t0}] = bi;
                } else {
                    bi = it->second;
                }
                ent.push_back({bi, {t - t0, {q, w[j]}}});
            }
        std::stable_sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        sb.assign(comb.size() + 1, 0);
        for (const auto& e : ent) sb[e.first + 1]++;
        for (size_t i = 0; i < comb.size(); ++i) sb[i + 1] += sb[i];
    }
    cudaFree(ctx->lblks_es);
    cudaFree(ctx->sbeg);
    cudaFree(ctx->sent);
    ctx->lblks_es = nullptr;
    ctx->sbeg = nullptr;
    ctx->sent = nullptr;
    ctx->nle_src = 0;
    cudaFree(ctx->dsrc);
    cudaFree(ctx->sdofs);
    cudaFree(ctx->sw);
    cudaFree(ctx->spdofs);
    ctx->spdofs = nullptr;
    ctx->dsrc = nullptr;
    ctx->sdofs = nullptr;
    ctx->sw = nullptr;
    int rc;
    if ((rc = upload(ctx, &ctx->dsrc, hs)) || (rc = upload(ctx, &ctx->sdofs, dofs)) || (rc = upload(ctx, &ctx->spdofs, pdofs)) ||
        (rc = upload_real(ctx, &ctx->sw, w)))
        return rc;
    if (!ent.empty()) {
        auto fill = [&](auto* dummy) {
            using R = std::remove_pointer_t<decltype(dummy)>;
            std::vector<SrcE<R>> se(ent.size());
            for (size_t i = 0; i < ent.size(); ++i)
                se[i] = SrcE<R>{ent[i].second.first, ent[i].second.second.first, (R)ent[i].second.second.second};
            SrcE<R>* d = nullptr;
            int r2 = upload(ctx, &d, se);
            ctx->sent = d;
            return r2;
        };
        if ((rc = upload(ctx, &ctx->lblks_es, comb)) || (rc = upload(ctx, &ctx->sbeg, sb)) ||
            (rc = ctx->precision == YGM_FP64 ? fill((double*)nullptr) : fill((float*)nullptr)))
            return rc;
        ctx->nle_src = (int)comb.size();
    }
    ctx->nsrc = n_src;
    ctx->src_cache.assign(src, src + n_src);
    return 0;
}

int ygm_step(ygm_ctx* ctx, int64_t n, double dt, const ygm_source* src, int32_t n_src) {
    if (ctx && ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (!ctx) return YGM_EINVAL;
    if (n < 0 || !(dt > 0) || !std::isfinite(dt)) return fail(ctx, YGM_EINVAL, "need n >= 0 and finite dt > 0");
    const std::vector<double>& wts = ctx->split_w;
    double wmax = 0.0;
    for (double w : wts) wmax = std::max(wmax, std::fabs(w));
    if (wmax * dt > ctx->S.tau_cfl * (1.0 + 1e-12))
        return fail(ctx, YGM_ECFL, "dt (times the largest splitting weight) exceeds the CFL bound 2/omega_max (Prop. stability)");
    if (n_src < 0 || (n_src > 0 && !src)) return fail(ctx, YGM_EINVAL, "bad source list");
    int rc = set_sources(ctx, src, n_src);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    void* b0 = ctx->b[ctx->cur];
    const double w1 = wts[0];
    if (!ctx->staggered) {
        // initial half step Phi^e_{dt/2} (Eq. YeeLeapfrog): b_{-1/2} = b_0 + dt/2 C Q1 e_0 (with a
        // composed splitting, the half of its first Strang sub-step, w_1 dt / 2)
        launch_qapply(ctx, ctx->x, false);
        launch_curl_b(ctx, ctx->x, b0, b0, -0.5 * w1 * dt);
        ctx->staggered = true;
        ctx->step_base = ctx->step;
        ctx->t_base = 0.0;
    } else if (dt != ctx->dt_prev) {
        // close the old staggering and reopen it with the new step (exact Strang composition)
        launch_qapply(ctx, ctx->x, false);
        launch_curl_b(ctx, ctx->x, b0, b0, 0.5 * w1 * ctx->dt_prev - 0.5 * w1 * dt);
        ctx->t_base += (double)(ctx->step - ctx->step_base) * ctx->dt_prev;
        ctx->step_base = ctx->step;
    }
    ctx->dt_prev = dt;
    // source amplitudes dt * s(t_{n+1/2}) for every step of this call (host, FP64); steps whose
    // amplitudes are all exactly 0.0 need no source launch (the update would add 0)
    // sub-steps of one step: kicks w_j dt at the sub-step midpoints, drifts (w_{j-1} + w_j) / 2 dt
    // (w_1 dt for the first: the pending half of the previous step's last sub-step, w_m = w_1, plus
    // its own leading half)
    const int m = (int)wts.size();
    std::vector<double> kick(m), drift(m), tmid(m);
    {
        double acc = 0.0;
        for (int j = 0; j < m; ++j) {
            kick[j] = wts[j];
            drift[j] = j == 0 ? wts[0] : 0.5 * (wts[j - 1] + wts[j]);
            tmid[j] = acc + 0.5 * wts[j];
            acc += wts[j];
        }
    }
    const double* amp_dev = nullptr;
    std::vector<char> src_on;
    if (ctx->nsrc && n > 0) {
        const int nsrc = ctx->nsrc;
        const size_t namp = (size_t)n * m * nsrc;
        int bsel = ctx->damp_cur;
        ctx->damp_cur ^= 1;
        CK(cudaEventSynchronize(ctx->damp_ev[bsel]));   // the buffer's previous readers are done
        if (ctx->damp_cap[bsel] < namp) {
            cudaFree(ctx->damp[bsel]);
            cudaFreeHost(ctx->hamp[bsel]);
            ctx->damp[bsel] = nullptr;
            ctx->hamp[bsel] = nullptr;
            CK(cudaMalloc((void**)&ctx->damp[bsel], namp * sizeof(double)));
            CK(cudaMallocHost((void**)&ctx->hamp[bsel], namp * sizeof(double)));
            ctx->damp_cap[bsel] = namp;
        }
        double* amp = ctx->hamp[bsel];
        src_on.assign((size_t)n * m, 0);
        for (int64_t i = 0; i < n; ++i)
            for (int j = 0; j < m; ++j) {
                const double t = ctx->t_base + ((double)(ctx->step + i - ctx->step_base) + tmid[j]) * dt;
                for (int q = 0; q < nsrc; ++q) {
                    const ygm_source& S0 = ctx->src_cache[q];
                    const double u = (t - S0.t0) / S0.sigma;
                    const double a = kick[j] * dt * S0.amp * std::exp(-u * u) * std::sin(S0.omega * (t - S0.t0));
                    amp[((size_t)i * m + j) * nsrc + q] = a;
                    if (a != 0.0) src_on[(size_t)i * m + j] = 1;
                }
            }
        CK(cudaMemcpyAsync(ctx->damp[bsel], amp, namp * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        amp_dev = ctx->damp[bsel];
    }
    if (ctx->energy_every && n > 0) {
        // the history grows to hold every record of this call (plus the two scratch records of
        // ygm_energy at its end), so no W_n is ever dropped
        const int64_t K = ctx->energy_every, first = (ctx->step + K - 1) / K, last = (ctx->step + n - 1) / K;
        const int64_t need = ctx->hist_n + (last - first + 1) + 2;
        if (need > ctx->hist_cap) {
            const int64_t cap = std::max<int64_t>(need, 2 * ctx->hist_cap);
            double* h = nullptr;
            CK(cudaMalloc((void**)&h, (size_t)cap * ctx->n_rhs * sizeof(double)));
            if (ctx->hist_n)
                CK(cudaMemcpyAsync(h, ctx->hist, (size_t)ctx->hist_n * ctx->n_rhs * sizeof(double), cudaMemcpyDeviceToDevice,
                                   ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            cudaFree(ctx->hist);
            ctx->hist = h;
            ctx->hist_cap = cap;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < m; ++j) {
            void* bo = ctx->b[ctx->cur];
            void* bn = ctx->b[ctx->cur ^ 1];
            const bool want_w = m == 1 && ctx->energy_every && ctx->step % ctx->energy_every == 0;
            launch_qapply(ctx, ctx->x, want_w);     // W_n needs e^T Q1 e over every row
            launch_curl_b(ctx, ctx->x, bo, bn, drift[j] * dt);
            if (want_w) launch_energy(ctx, ctx->e, ctx->x, bn, bo, ctx->hist + (size_t)ctx->n_rhs * ctx->hist_n++);
            const size_t si = (size_t)i * m + j;
            launch_curlT_e(ctx, bn, ctx->e, kick[j] * dt, amp_dev && src_on[si] ? amp_dev + si * ctx->nsrc : nullptr);
            ctx->cur ^= 1;
        }
        ctx->step++;
    }
    if (amp_dev) CK(cudaEventRecord(ctx->damp_ev[ctx->damp_cur ^ 1], ctx->stream));
    CK(cudaGetLastError());
    return YGM_OK;
}

int ygm_set_splitting(ygm_ctx* ctx, int32_t order) {
    if (!ctx) return YGM_EINVAL;
    if (ctx->staggered)
        return fail(ctx, YGM_EINVAL, "set the splitting before the first step (or after ygm_set_state / ygm_project_E)");
    if (order == 2) {
        ctx->split_w.assign(1, 1.0);
    } else if (order == 4) {
        if (ctx->energy_every)
            return fail(ctx, YGM_EINVAL, "W_n is the invariant of the Strang leapfrog only: energy_every must be 0 for order 4");
        const double c = std::cbrt(2.0), w1 = 1.0 / (2.0 - c);
        ctx->split_w = {w1, -c * w1, w1};
    } else {
        return fail(ctx, YGM_EINVAL, "splitting order must be 2 or 4");
    }
    return YGM_OK;
}

int ygm_energy(ygm_ctx* ctx, double* W, double* Htilde) {
    if (ctx && ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (!ctx || !W) return fail(ctx, YGM_EINVAL, "NULL argument");
    const size_t nb = ctx->S.L.N2 * ctx->n_rhs * ctx->rs;
    const int R = ctx->n_rhs;
    double* dout = ctx->hist + (size_t)(ctx->hist_cap - 2) * R;   // two scratch records at the end of the history
    void* bo = ctx->b[ctx->cur];
    launch_qapply(ctx, ctx->x, true);
    if (ctx->staggered) {
        const double tw = ctx->split_w[0] * ctx->dt_prev;   // the (first) Strang sub-step
        CK(cudaMemcpyAsync(ctx->bscr, bo, nb, cudaMemcpyDeviceToDevice, ctx->stream));
        launch_curl_b(ctx, ctx->x, bo, ctx->bscr, tw);
        launch_energy(ctx, ctx->e, ctx->x, ctx->bscr, bo, dout);
        launch_curl_b(ctx, ctx->x, bo, ctx->bscr, 0.5 * tw);
        launch_energy(ctx, ctx->e, ctx->x, ctx->bscr, ctx->bscr, dout + R);
    } else {
        // not yet staggered: b is synchronised, W is reported as H~
        launch_energy(ctx, ctx->e, ctx->x, bo, bo, dout);
        launch_energy(ctx, ctx->e, ctx->x, bo, bo, dout + R);
    }
    std::vector<double> h(2 * (size_t)R);
    CK(cudaMemcpyAsync(h.data(), dout, 2 * (size_t)R * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::copy(h.begin(), h.begin() + R, W);
    if (Htilde) std::copy(h.begin() + R, h.end(), Htilde);
    return check_device_flags(ctx);
}

int ygm_energy_history(ygm_ctx* ctx, double* out, int64_t max_count, int64_t* count) {
    if (ctx && ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (!ctx || !count) return fail(ctx, YGM_EINVAL, "NULL argument");
    int64_t c = std::min<int64_t>(ctx->hist_n, max_count);
    if (c > 0 && out)
        CK(cudaMemcpyAsync(out, ctx->hist, (size_t)c * ctx->n_rhs * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *count = c;
    return YGM_OK;
}

int ygm_time(const ygm_ctx* ctx, int64_t* step, double* t) {
    if (!ctx) return YGM_EINVAL;
    if (step) *step = ctx->step;
    if (t) *t = ctx->t_base + (double)(ctx->step - ctx->step_base) * ctx->dt_prev;
    return YGM_OK;
}

int ygm_export_q1(const ygm_ctx* ctx, int64_t* rowptr, int64_t* colind, double* val) {
    if (!ctx || !rowptr || !colind || !val) return YGM_EINVAL;
    const auto& Q = ctx->S.Q1;
    std::copy(Q.ptr.begin(), Q.ptr.end(), rowptr);
    std::copy(Q.col.begin(), Q.col.end(), colind);
    std::copy(Q.val.begin(), Q.val.end(), val);
    return YGM_OK;
}

// Device copies of a new Q1 (box-indexed, and the full-row or upper-triangle lattice copy the
// step reads): uploaded into fresh buffers first; the old ones are freed and replaced only once
// every upload succeeded, so a failed refresh leaves the context stepping the previous Q1.
static int refresh_q1_device(ygm_ctx* ctx) {
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    void *q = nullptr, *qf = nullptr, *qsd = nullptr;
    int rc = upload_real(ctx, &q, ctx->S.qvals);
    if (!rc && !ctx->use_sym) rc = upload_real(ctx, &qf, ctx->S.qfull);
    if (!rc && ctx->use_sym) rc = upload_real(ctx, &qsd, ctx->S.qsym);
    if (rc) {
        cudaFree(q);
        cudaFree(qf);
        cudaFree(qsd);
        return rc;
    }
    cudaFree(ctx->q);
    cudaFree(ctx->qf);
    cudaFree(ctx->qsd);
    ctx->q = q;
    ctx->qf = qf;
    ctx->qsd = qsd;
    return 0;
}

// A Q1 update that failed its SPD check: put the previous Q1 back into the host set-up (the
// device copies were not touched) and keep the error message.
static int restore_q1(ygm_ctx* ctx, ygm::Csr&& old, int code) {
    const std::string msg = code == YGM_ENOTSPD ? ctx->S.err : ctx->err;   // set-up check, or a failed upload
    ctx->S.Q1 = std::move(old);
    ygm::repack_q1(ctx->S, 0);
    return fail(ctx, code, msg);
}

int ygm_set_q1(ygm_ctx* ctx, const int64_t* rowptr, const int64_t* colind, const double* val) {
    if (!ctx || !rowptr || !colind || !val) return fail(ctx, YGM_EINVAL, "NULL argument");
    ygm::Csr old = ctx->S.Q1;
    int rc = ygm::install_q1(ctx->S, rowptr, colind, val, 0);
    if (rc == -1) return fail(ctx, YGM_EINVAL, ctx->S.err);
    if (rc) return restore_q1(ctx, std::move(old), YGM_ENOTSPD);
    if (!ctx->host_only && (rc = refresh_q1_device(ctx))) return restore_q1(ctx, std::move(old), rc);
    return YGM_OK;
}

int ygm_spai_op(ygm_ctx* ctx, const double* V, int32_t n_probe, double lambda, int32_t max_iter, double tol,
                int32_t* iters, double* rel_residual) {
    if (!ctx) return YGM_EINVAL;
    int it = 0;
    double rr = 0.0;
    ygm::Csr old = ctx->S.Q1;
    int rc = ygm::spai_op(ctx->S, V, n_probe, lambda, max_iter, tol, 0, &it, &rr);
    if (iters) *iters = it;
    if (rel_residual) *rel_residual = rr;
    if (rc == -1 || rc == -2) return fail(ctx, rc == -1 ? YGM_EINVAL : YGM_ETIMEOUT, ctx->S.err);
    if (rc) return restore_q1(ctx, std::move(old), YGM_ENOTSPD);
    if (!ctx->host_only && (rc = refresh_q1_device(ctx))) return restore_q1(ctx, std::move(old), rc);
    return YGM_OK;
}

int ygm_cavity_modes(ygm_ctx* ctx, int32_t count, double* V, double* omega_sq, int32_t max_iter, double tol,
                     int32_t* iters) {
    if (!ctx) return YGM_EINVAL;
    int it = 0;
    int rc = ygm::cavity_modes(ctx->S, count, V, omega_sq, max_iter, tol, 0, &it);
    if (iters) *iters = it;
    if (rc) return fail(ctx, rc == -1 ? YGM_EINVAL : rc == -2 ? YGM_ETIMEOUT : YGM_EINVAL, ctx->S.err);
    return YGM_OK;
}

int ygm_q1_vjp(ygm_ctx* ctx, const double* q1bar, double* grad_eps) {
    if (!ctx || !q1bar || !grad_eps) return fail(ctx, YGM_EINVAL, "NULL argument");
    const int rc = ygm::q1_vjp(ctx->S, q1bar, grad_eps, 0);
    if (rc == -1) return fail(ctx, YGM_EINVAL, "ygm_q1_vjp: the Q1 pattern is not symmetric");
    if (rc) return fail(ctx, YGM_ENOTSPD, "ygm_q1_vjp: a column normal matrix is not SPD");
    return YGM_OK;
}

int ygm_step_noalloc(ygm_ctx* ctx, void* e, const void* b_in, void* b_out, double dt) {
    if (!ctx || !e || !b_in || !b_out) return fail(ctx, YGM_EINVAL, "NULL argument");
    const size_t need = (size_t)ctx->S.L.N1 * ctx->n_rhs * ctx->rs;
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(ctx, YGM_EINVAL,
                    "ygm_step_noalloc: N1 * n_rhs * sizeof(real) = " + std::to_string(need) +
                        " bytes exceeds the fixed 16 MiB scratch (use ygm_step)");
    if (ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (ctx->n_rhs != 1) return fail(ctx, YGM_EINVAL, "ygm_step_noalloc: contexts with n_rhs > 1 are not supported");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, YGM_EINVAL, "need finite dt > 0");
    if (dt > ctx->S.tau_cfl * (1.0 + 1e-12))
        return fail(ctx, YGM_ECFL, "dt exceeds the CFL bound 2/omega_max (Prop. stability)");
    if (ctx->device < 0 || ctx->device >= 256) return fail(ctx, YGM_EINVAL, "device ordinal out of range");
    CK(cudaSetDevice(ctx->device));
    void* x = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mutex);
        if (!g_noalloc_addr[ctx->device]) {
            void* p = nullptr;
            CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_addr[ctx->device] = p;
        }
        x = g_noalloc_addr[ctx->device];
    }
    // x = Q1 e (every element of x is written, so the scratch needs no clearing)
    const size_t smem = (size_t)ctx->max_slots * (2 * sizeof(long long) + 8 * sizeof(int));
    if (ctx->nqblocks) {
        if (ctx->precision == YGM_FP64)
            k_qapply_b<double><<<ctx->nqblocks, ctx->qthreads, smem, ctx->stream>>>(
                ctx->c1, ctx->qslots, ctx->qblocks, ctx->max_slots, (const double*)ctx->q, (const double*)e, (double*)x);
        else
            k_qapply_b<float><<<ctx->nqblocks, ctx->qthreads, smem, ctx->stream>>>(
                ctx->c1, ctx->qslots, ctx->qblocks, ctx->max_slots, (const float*)ctx->q, (const float*)e, (float*)x);
    }
    // b_out = b_in - dt C x ; e += dt C^T M2 b_out
    if (ctx->nbblocks) {
        if (ctx->precision == YGM_FP64)
            k_curl_b_b<double><<<ctx->nbblocks, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->c2, ctx->terms, ctx->bblocks,
                                                                         (const double*)x, (const double*)b_in,
                                                                         (double*)b_out, dt);
        else
            k_curl_b_b<float><<<ctx->nbblocks, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->c2, ctx->terms, ctx->bblocks,
                                                                        (const float*)x, (const float*)b_in,
                                                                        (float*)b_out, (float)dt);
    }
    if (ctx->pterms) {
        const int mt = ctx->max_terms;
        const size_t smem_e = (size_t)mt * sizeof(long long) + (size_t)(mt + (mt & 1)) * ctx->rs + (size_t)mt * 6 * sizeof(int);
        if (ctx->neblocks) {
            if (ctx->precision == YGM_FP64)
                k_curlT_e_b<double><<<ctx->neblocks, BLOCK, smem_e, ctx->stream>>>(
                    ctx->c1, ctx->pbeg, (const PTerm<double>*)ctx->pterms, ctx->eblocks, mt, (const double*)b_out, (double*)e, dt,
                    nullptr, ctx->pg);
            else
                k_curlT_e_b<float><<<ctx->neblocks, BLOCK, smem_e, ctx->stream>>>(
                    ctx->c1, ctx->pbeg, (const PTerm<float>*)ctx->pterms, ctx->eblocks, mt, (const float*)b_out, (float*)e,
                    (float)dt, nullptr, ctx->pg);
        }
    } else {
        dim3 g((ctx->nrowsE + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
        if (ctx->precision == YGM_FP64)
            k_curlT_e<double><<<g, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->rowsE, ctx->nrowsE, (const double*)ctx->W,
                                                            (const double*)b_out, (const double*)ctx->inv_mu, (double*)e, dt,
                                                            nullptr, ctx->pg);
        else
            k_curlT_e<float><<<g, BLOCK, 0, ctx->stream>>>(ctx->tb, ctx->rowsE, ctx->nrowsE, (const float*)ctx->W,
                                                           (const float*)b_out, (const float*)ctx->inv_mu, (float*)e,
                                                           (float)dt, nullptr, ctx->pg);
    }
    ctx->launches += 3;
    CK(cudaGetLastError());
    return YGM_OK;
}

// ---------------------------------------------------------------------- uneven batch
}  // extern "C"

struct ygm_batch {
    std::vector<ygm_ctx*> cav;
    int device = 0, precision = YGM_FP32;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    void* dcavs = nullptr;               // BCav<real>[count]
    int2* items = nullptr;
    size_t items_cap = 0;
    int nA = 0, nB = 0, nC = 0;
    size_t smem = 0;
    int max_per_sm = 1, nsm = 0;
    double* amp = nullptr;
    size_t amp_cap = 0;
    unsigned* bar = nullptr;
    int* err = nullptr;
    int ctas_per_sm = 1, order = 1;      // launch shape and work order (ygm_batch_tune)
    long long wait_cap = 1LL << 24;      // polls of a grid-barrier wait before it gives up
    cudaGraphExec_t gexec = nullptr;
    int64_t g_steps = -1;
    int g_grid = -1, g_order = -1;
    std::string errmsg;
};

static int bfail(ygm_batch* B, int code, const std::string& m) {
    B->errmsg = m;
    return code;
}
#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess) return bfail(B, YGM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// Work items of the three phases.  order 0: cavity by cavity; order 1: Q1-apply items sorted by
// their stencil length (longest first) and every phase interleaved across cavities, so that the
// static round-robin over CTAs spreads the heavy (order 3) cavities.
static int batch_items(ygm_batch* B) {
    std::vector<int2> A, Bb, Cc;
    const int nc = (int)B->cav.size();
    std::vector<std::pair<int, int2>> a;
    for (int c = 0; c < nc; ++c) {
        ygm_ctx* x = B->cav[c];
        std::vector<SBlk> sb(x->nsblks_act);
        if (x->nsblks_act) BCK(cudaMemcpy(sb.data(), x->sblks, sb.size() * sizeof(SBlk), cudaMemcpyDeviceToHost));
        for (int i = 0; i < x->nsblks_act; ++i) {
            const auto& st = x->S.st_begin;
            a.push_back({st[sb[i].cls + 1] - st[sb[i].cls], make_int2(c, i)});
        }
    }
    auto inter = [&](auto count) {
        std::vector<int2> out;
        int mx = 0;
        for (int c = 0; c < nc; ++c) mx = std::max(mx, count(c));
        if (B->order == 0) {
            for (int c = 0; c < nc; ++c)
                for (int i = 0; i < count(c); ++i) out.push_back(make_int2(c, i));
        } else {
            for (int i = 0; i < mx; ++i)
                for (int c = 0; c < nc; ++c)
                    if (i < count(c)) out.push_back(make_int2(c, i));
        }
        return out;
    };
    if (B->order == 0) {
        for (auto& v : a) A.push_back(v.second);
    } else {
        std::stable_sort(a.begin(), a.end(), [](const auto& u, const auto& v) { return u.first > v.first; });
        for (auto& v : a) A.push_back(v.second);
    }
    Bb = inter([&](int c) { return B->cav[c]->nlb; });
    Cc = inter([&](int c) { return B->cav[c]->lblks_es ? B->cav[c]->nle_src : B->cav[c]->nle; });
    std::vector<int2> all(A);
    all.insert(all.end(), Bb.begin(), Bb.end());
    all.insert(all.end(), Cc.begin(), Cc.end());
    if (all.size() > B->items_cap) {
        cudaFree(B->items);
        B->items = nullptr;
        BCK(cudaMalloc((void**)&B->items, all.size() * sizeof(int2)));
        B->items_cap = all.size();
    }
    if (!all.empty()) BCK(cudaMemcpy(B->items, all.data(), all.size() * sizeof(int2), cudaMemcpyHostToDevice));
    B->nA = (int)A.size();
    B->nB = (int)Bb.size();
    B->nC = (int)Cc.size();
    return 0;
}

template <typename real>
static BCav<real> bcav_of(ygm_ctx* x, double dt) {
    BCav<real> c{};
    c.c1 = x->c1;
    c.c2 = x->c2;
    c.soff2 = x->soff2;
    c.sg = x->sg;
    c.pg = x->pg;
    c.qs = (const real*)x->qsd;
    c.ep = (real*)x->ep;
    c.x = (real*)x->x;
    c.xp = (real*)x->xp;
    c.bp = (real*)x->bp;
    c.b0 = (real*)x->b[0];
    c.b1 = (real*)x->b[1];
    c.e = (real*)x->e;
    c.cterms = x->cterms;
    c.pbeg = x->pbeg;
    c.wterms = (const WTermL<real>*)x->wterms;
    c.blkA = x->sblks;
    c.blkB = x->lblks_b;
    c.blkC = x->lblks_es ? x->lblks_es : x->lblks_e;
    c.sbeg = x->lblks_es ? x->sbeg : nullptr;
    c.sent = (const SrcE<real>*)x->sent;
    c.tau = split_tau<real>(dt);
    c.cur0 = x->cur;
    return c;
}

template <typename real>
static int batch_launch(ygm_batch* B, int64_t nsteps, bool graph) {
    const int ncav = (int)B->cav.size();
    const int grid = B->nsm * B->ctas_per_sm;
    int ns = (int)nsteps;
    void* args[] = {&B->dcavs, &B->items, &B->nA, &B->nB, &B->nC, &ns, (void*)&ncav, &B->amp, &B->bar, &B->err, &B->wait_cap};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(SBLOCK);
    cfg.dynamicSmemBytes = B->smem;
    cfg.stream = B->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    auto issue = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(B->bar, 0, 2 * sizeof(unsigned), B->stream);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelExC(&cfg, (const void*)k_batch<real>, args);
    };
    if (!graph) {
        BCK(issue());
        return 0;
    }
    if (!B->gexec || B->g_steps != nsteps || B->g_grid != grid || B->g_order != B->order) {
        if (B->gexec) cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = issue();
        const cudaError_t ce = cudaStreamEndCapture(B->stream, &g);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(B, YGM_ECUDA, std::string("capturing the batch launch: ") + cudaGetErrorString(le != cudaSuccess ? le : ce));
        }
        const cudaError_t ie = cudaGraphInstantiate(&B->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return bfail(B, YGM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        B->g_steps = nsteps;
        B->g_grid = grid;
        B->g_order = B->order;
    }
    BCK(cudaGraphLaunch(B->gexec, B->stream));
    return 0;
}

extern "C" {

int ygm_batch_create(ygm_ctx* const* cavities, int32_t count, ygm_batch** out) {
    if (!out) return YGM_EINVAL;
    *out = nullptr;
    if (!cavities || count < 1) return YGM_EINVAL;
    ygm_batch* B = new (std::nothrow) ygm_batch();
    if (!B) return YGM_ENOMEM;
    auto bad = [&](int code, const std::string& m) {
        std::lock_guard<std::mutex> lk(g_err_mutex);
        g_create_err = m;
        delete B;
        return code;
    };
    for (int i = 0; i < count; ++i) {
        ygm_ctx* x = cavities[i];
        if (!x) return bad(YGM_EINVAL, "NULL context");
        if (x->host_only) return bad(YGM_ENODEV, "host-only context in the batch");
        if (!x->use_sym || x->n_rhs != 1 || !x->wterms || !x->nle || x->tc_passes || x->split_w.size() != 1)
            return bad(YGM_EINVAL, "batch members must be one-column FP32/FP64 Strang contexts with uniform mu on the lattice path");
        if (x->device != cavities[0]->device || x->precision != cavities[0]->precision)
            return bad(YGM_EINVAL, "batch members must share the device and the precision");
        B->cav.push_back(x);
    }
    B->device = cavities[0]->device;
    B->precision = cavities[0]->precision;
    B->stream = cavities[0]->stream;
    if (cudaSetDevice(B->device) != cudaSuccess) return bad(YGM_ECUDA, "cudaSetDevice failed");
    for (ygm_ctx* x : B->cav) {
        const size_t rsz = B->precision == YGM_FP64 ? sizeof(WTermL<double>) : sizeof(WTermL<float>);
        B->smem = std::max(B->smem, std::max((size_t)(x->max_ns + 8) * sizeof(int2), (size_t)x->max_terms * rsz));
    }
    if (B->smem > 48 * 1024) return bad(YGM_EINVAL, "batch: stencil tables exceed 48 KB of shared memory");
    int nb = 0;
    const cudaError_t oe = B->precision == YGM_FP64
                               ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<double>, SBLOCK, B->smem)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<float>, SBLOCK, B->smem);
    if (oe != cudaSuccess || nb < 1) return bad(YGM_ECUDA, "batch: occupancy query failed");
    B->max_per_sm = nb;
    B->ctas_per_sm = std::min(nb, 4);
    if (cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess)
        return bad(YGM_ECUDA, "batch: SM count query failed");
    const size_t cbytes = (B->precision == YGM_FP64 ? sizeof(BCav<double>) : sizeof(BCav<float>)) * count;
    if (cudaMalloc(&B->dcavs, cbytes) != cudaSuccess || cudaMalloc((void**)&B->bar, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void**)&B->err, sizeof(int)) != cudaSuccess || cudaMemset(B->err, 0, sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming) != cudaSuccess) {
        ygm_batch_destroy(B);
        std::lock_guard<std::mutex> lk(g_err_mutex);
        g_create_err = "batch: device allocation failed";
        return YGM_ENOMEM;
    }
    if (int rc = batch_items(B)) {
        std::string m = B->errmsg;
        ygm_batch_destroy(B);
        std::lock_guard<std::mutex> lk(g_err_mutex);
        g_create_err = m;
        return rc;
    }
    *out = B;
    return YGM_OK;
}

int ygm_batch_step(ygm_batch* B, int64_t nsteps, const double* dt, const ygm_source* src, int32_t use_graph) {
    if (!B || !dt || nsteps < 0) return B ? bfail(B, YGM_EINVAL, "need dt[] and nsteps >= 0") : YGM_EINVAL;
    const int nc = (int)B->cav.size();
    for (int i = 0; i < nc; ++i) {
        ygm_ctx* x = B->cav[i];
        if (!(dt[i] > 0) || !std::isfinite(dt[i])) return bfail(B, YGM_EINVAL, "dt must be finite and > 0");
        if (dt[i] > x->S.tau_cfl * (1.0 + 1e-12))
            return bfail(B, YGM_ECFL, "cavity " + std::to_string(i) + ": dt exceeds its CFL bound (Prop. stability)");
    }
    BCK(cudaSetDevice(B->device));
    bool relist = false;
    for (int i = 0; i < nc; ++i) {
        ygm_ctx* x = B->cav[i];
        ygm_source s1{};
        if (src) {
            s1 = src[i];
            s1.rhs = 0;
        }
        const bool had = x->lblks_es != nullptr;
        const int nsb = x->nle_src;
        if (int rc = set_sources(x, src ? &s1 : nullptr, src ? 1 : 0))
            return bfail(B, rc, "cavity " + std::to_string(i) + ": " + x->err);
        relist |= had != (x->lblks_es != nullptr) || nsb != x->nle_src;
        // staggering of each cavity on its own stream (as ygm_step), then ordered before the batch
        void* b0 = x->b[x->cur];
        if (!x->staggered) {
            launch_qapply(x, x->x, false);
            launch_curl_b(x, x->x, b0, b0, -0.5 * dt[i]);
            x->staggered = true;
            x->step_base = x->step;
            x->t_base = 0.0;
        } else if (dt[i] != x->dt_prev) {
            launch_qapply(x, x->x, false);
            launch_curl_b(x, x->x, b0, b0, 0.5 * x->dt_prev - 0.5 * dt[i]);
            x->t_base += (double)(x->step - x->step_base) * x->dt_prev;
            x->step_base = x->step;
        }
        x->dt_prev = dt[i];
        if (x->stream != B->stream) {
            BCK(cudaEventRecord(B->ev, x->stream));
            BCK(cudaStreamWaitEvent(B->stream, B->ev, 0));
        }
    }
    if (relist)
        if (int rc = batch_items(B)) return rc;
    if (nsteps == 0) return YGM_OK;
    // per-step, per-cavity source amplitudes dt s(t_{n+1/2}) (host FP64)
    const size_t namp = (size_t)nsteps * nc;
    std::vector<double> amp(namp, 0.0);
    for (int i = 0; i < nc; ++i) {
        ygm_ctx* x = B->cav[i];
        if (!x->nsrc) continue;
        const ygm_source& s0 = x->src_cache[0];
        for (int64_t st = 0; st < nsteps; ++st) {
            const double t = x->t_base + ((double)(x->step + st - x->step_base) + 0.5) * dt[i];
            const double u = (t - s0.t0) / s0.sigma;
            amp[(size_t)st * nc + i] = dt[i] * s0.amp * std::exp(-u * u) * std::sin(s0.omega * (t - s0.t0));
        }
    }
    BCK(cudaStreamSynchronize(B->stream));   // the previous launch no longer reads amp / dcavs
    if (namp > B->amp_cap) {
        cudaFree(B->amp);
        B->amp = nullptr;
        BCK(cudaMalloc((void**)&B->amp, namp * sizeof(double)));
        B->amp_cap = namp;
        if (B->gexec) cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    BCK(cudaMemcpy(B->amp, amp.data(), namp * sizeof(double), cudaMemcpyHostToDevice));
    int rc;
    if (B->precision == YGM_FP64) {
        std::vector<BCav<double>> cv(nc);
        for (int i = 0; i < nc; ++i) cv[i] = bcav_of<double>(B->cav[i], dt[i]);
        BCK(cudaMemcpy(B->dcavs, cv.data(), cv.size() * sizeof(cv[0]), cudaMemcpyHostToDevice));
        rc = batch_launch<double>(B, nsteps, use_graph != 0);
    } else {
        std::vector<BCav<float>> cv(nc);
        for (int i = 0; i < nc; ++i) cv[i] = bcav_of<float>(B->cav[i], dt[i]);
        BCK(cudaMemcpy(B->dcavs, cv.data(), cv.size() * sizeof(cv[0]), cudaMemcpyHostToDevice));
        rc = batch_launch<float>(B, nsteps, use_graph != 0);
    }
    if (rc) return rc;
    for (ygm_ctx* x : B->cav) {
        x->cur ^= (int)(nsteps & 1);
        x->step += nsteps;
        x->launches += 1;
        if (x->stream != B->stream) {
            BCK(cudaEventRecord(B->ev, B->stream));
            BCK(cudaStreamWaitEvent(x->stream, B->ev, 0));
        }
    }
    return YGM_OK;
}

int ygm_batch_status(ygm_batch* B) {
    if (!B) return YGM_EINVAL;
    int h = 0;
    BCK(cudaStreamSynchronize(B->stream));
    BCK(cudaMemcpy(&h, B->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return bfail(B, YGM_ETIMEOUT, "batch: a grid barrier gave up waiting (not every CTA was resident)");
    return YGM_OK;
}

int ygm_batch_tune(ygm_batch* B, int32_t trial_steps, const double* dt, const ygm_source* src, int32_t* ctas_per_sm,
                   int32_t* order, double* ms_per_step) {
    if (!B || !dt || trial_steps < 1) return B ? bfail(B, YGM_EINVAL, "need dt[] and trial_steps >= 1") : YGM_EINVAL;
    BCK(cudaSetDevice(B->device));
    // save every cavity's state (the trials advance it), restore it after each trial
    struct Saved {
        std::vector<void*> buf;
        int cur;
        bool stag;
        int64_t step, step_base;
        double t_base, dt_prev;
    };
    std::vector<Saved> sv(B->cav.size());
    auto cleanup = [&]() {
        for (auto& s0 : sv)
            for (void* p : s0.buf) cudaFree(p);
    };
    for (size_t i = 0; i < B->cav.size(); ++i) {
        ygm_ctx* x = B->cav[i];
        BCK(cudaStreamSynchronize(x->stream));
        const size_t sz[4] = {x->S.L.N1 * x->rs, x->S.L.N2 * x->rs, x->S.L.N2 * x->rs, (size_t)x->n1pad * x->rs};
        void* src4[4] = {x->e, x->b[0], x->b[1], x->ep};
        for (int j = 0; j < 4; ++j) {
            void* p = nullptr;
            if (cudaMalloc(&p, sz[j]) != cudaSuccess) {
                cleanup();
                return bfail(B, YGM_ENOMEM, "batch tune: saving a state failed");
            }
            sv[i].buf.push_back(p);
            BCK(cudaMemcpy(p, src4[j], sz[j], cudaMemcpyDeviceToDevice));
        }
        sv[i].cur = x->cur;
        sv[i].stag = x->staggered;
        sv[i].step = x->step;
        sv[i].step_base = x->step_base;
        sv[i].t_base = x->t_base;
        sv[i].dt_prev = x->dt_prev;
    }
    auto restore = [&]() -> int {
        for (size_t i = 0; i < B->cav.size(); ++i) {
            ygm_ctx* x = B->cav[i];
            BCK(cudaStreamSynchronize(B->stream));
            const size_t sz[4] = {x->S.L.N1 * x->rs, x->S.L.N2 * x->rs, x->S.L.N2 * x->rs, (size_t)x->n1pad * x->rs};
            void* dst4[4] = {x->e, x->b[0], x->b[1], x->ep};
            for (int j = 0; j < 4; ++j) BCK(cudaMemcpy(dst4[j], sv[i].buf[j], sz[j], cudaMemcpyDeviceToDevice));
            x->cur = sv[i].cur;
            x->staggered = sv[i].stag;
            x->step = sv[i].step;
            x->step_base = sv[i].step_base;
            x->t_base = sv[i].t_base;
            x->dt_prev = sv[i].dt_prev;
        }
        return 0;
    };
    double best = 1e300;
    int bc = B->ctas_per_sm, bo = B->order;
    cudaEvent_t a, z;
    BCK(cudaEventCreate(&a));
    BCK(cudaEventCreate(&z));
    for (int o = 0; o < 2; ++o)
        for (int c = 1; c <= std::min(B->max_per_sm, 4); ++c) {
            B->order = o;
            B->ctas_per_sm = c;
            int rc = batch_items(B);
            if (!rc) rc = ygm_batch_step(B, 1, dt, src, 0);   // staggering and sources outside the timed launch
            if (!rc) rc = cudaEventRecord(a, B->stream) == cudaSuccess ? 0 : YGM_ECUDA;
            if (!rc) rc = ygm_batch_step(B, trial_steps, dt, src, 0);
            if (!rc) rc = cudaEventRecord(z, B->stream) == cudaSuccess ? 0 : YGM_ECUDA;
            if (!rc) rc = ygm_batch_status(B);
            float ms = 0.f;
            if (!rc) rc = cudaEventElapsedTime(&ms, a, z) == cudaSuccess ? 0 : YGM_ECUDA;
            const int rr = restore();
            if (rc || rr) {
                cudaEventDestroy(a);
                cudaEventDestroy(z);
                cleanup();
                return rc ? rc : rr;
            }
            if (ms < best) {
                best = ms;
                bc = c;
                bo = o;
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    cleanup();
    B->ctas_per_sm = bc;
    B->order = bo;
    if (int rc = batch_items(B)) return rc;
    if (ctas_per_sm) *ctas_per_sm = bc;
    if (order) *order = bo;
    if (ms_per_step) *ms_per_step = best / trial_steps;
    return YGM_OK;
}

int ygm_batch_wait_limit(ygm_batch* B, int64_t polls) {
    if (!B || polls < 0) return YGM_EINVAL;
    B->wait_cap = polls;
    if (B->gexec) cudaGraphExecDestroy(B->gexec);   // the cap is a kernel argument of the captured launch
    B->gexec = nullptr;
    return YGM_OK;
}

int ygm_batch_status_clear(ygm_batch* B) {
    if (!B) return YGM_EINVAL;
    BCK(cudaStreamSynchronize(B->stream));
    BCK(cudaMemset(B->err, 0, sizeof(int)));
    return YGM_OK;
}

const char* ygm_batch_last_error(const ygm_batch* B) { return B ? B->errmsg.c_str() : ""; }

void ygm_batch_destroy(ygm_batch* B) {
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    cudaFree(B->dcavs);
    cudaFree(B->items);
    cudaFree(B->amp);
    cudaFree(B->bar);
    cudaFree(B->err);
    if (B->ev) cudaEventDestroy(B->ev);
    delete B;
}

}  // extern "C"

// ---------------------------------------------------------------------- adjoint (one column)
// Host tables of the probe region: its tets' DoFs, the region mass operators as CSR, the padded
// index of every 1-form DoF.  Sums over tets run in tet order (deterministic).
struct RegionOps {
    std::vector<int> tets, d1, d2;            // region tets; their n1 / n2a global DoFs (-1: none)
    std::vector<double> epsr, imur;
    std::vector<int> g_rows, g_ptr, g_col;    // C^T M2^R on the rows it touches
    std::vector<double> g_val;
    std::vector<int> m_ptr, m_col;            // M1^R over all N1 rows
    std::vector<double> m_val;
};
static void build_region(const ygm_ctx* ctx, const uint8_t* region, RegionOps& R) {
    const ygm::Setup& S = ctx->S;
    const ygm::Lattice& L = S.L;
    const int64_t T = 6LL * L.n * L.n * L.n;
    const int n1 = L.n1, n2a = L.n2a;
    std::vector<int64_t> g1(n1), g2(L.n2);
    std::map<std::pair<int, int>, double> G, M;
    for (int64_t t = 0; t < T; ++t) {
        if (!region[t]) continue;
        L.tet_dofs1(t, g1.data());
        L.tet_dofs2(t, g2.data());
        R.tets.push_back((int)t);
        const double eps = S.eps.empty() ? 1.0 : S.eps[t], imu = S.mu.empty() ? 1.0 : 1.0 / S.mu[t];
        R.epsr.push_back(eps);
        R.imur.push_back(imu);
        for (int a = 0; a < n1; ++a) R.d1.push_back((int)g1[a]);
        for (int r = 0; r < n2a; ++r) R.d2.push_back((int)g2[L.act2[r]]);
        for (int a = 0; a < n1; ++a) {
            if (g1[a] < 0) continue;
            for (int r = 0; r < n2a; ++r) {
                const int64_t j = g2[L.act2[r]];
                if (j >= 0) G[{(int)g1[a], (int)j}] += S.Wloc[(size_t)a * n2a + r] * imu;
            }
            for (int c = 0; c < n1; ++c)
                if (g1[c] >= 0) M[{(int)g1[a], (int)g1[c]}] += S.M1loc[(size_t)a * n1 + c] * eps;
        }
    }
    R.g_ptr.push_back(0);
    int last = -1;
    for (const auto& kv : G) {
        if (kv.first.first != last) {
            if (last >= 0) R.g_ptr.push_back((int)R.g_col.size());
            R.g_rows.push_back(kv.first.first);
            last = kv.first.first;
        }
        R.g_col.push_back(kv.first.second);
        R.g_val.push_back(kv.second);
    }
    if (last >= 0) R.g_ptr.push_back((int)R.g_col.size());
    R.m_ptr.assign(L.N1 + 1, 0);
    for (const auto& kv : M) R.m_ptr[kv.first.first + 1]++;
    for (int64_t i = 0; i < L.N1; ++i) R.m_ptr[i + 1] += R.m_ptr[i];
    for (const auto& kv : M) {
        R.m_col.push_back(kv.first.second);
        R.m_val.push_back(kv.second);
    }
}

// dL/dQ1 on the CSR pattern of Q1 from the pair sums S[i, s] of the upper-triangle lattice:
// qbar_ij = qbar_ji = S / 2 (the symmetric part is what the SPAI derivative uses).
template <typename real>
static void pairs_to_csr(const ygm::Setup& S, const std::vector<real>& Sv, std::vector<double>& qbar) {
    const ygm::Lattice& L = S.L;
    const size_t nc = L.c1.size();
    std::vector<std::map<std::array<int, 4>, int>> up(nc);   // (nbr class, d) -> upper slot
    for (size_t c = 0; c < nc; ++c)
        for (int k = S.st_begin[c]; k < S.st_begin[c + 1]; ++k) {
            const auto& st = S.st_slots[k];
            if (st.upper) up[c][{st.cls, st.d[0], st.d[1], st.d[2]}] = st.slot;
        }
    qbar.assign(S.Q1.col.size(), 0.0);
    const int NX = S.qs_nx, NY = S.qs_ny;
    auto at = [&](int c, int slot, const int v[3]) {
        return S.qs_base[c] + (int64_t)slot * S.qs_vol + ((int64_t)v[2] * NY + v[1]) * NX + v[0];
    };
    for (int64_t i = 0; i < L.N1; ++i) {
        int ci, vi[3];
        L.decode1(i, &ci, vi);
        for (int64_t k = S.Q1.ptr[i]; k < S.Q1.ptr[i + 1]; ++k) {
            int cj, vj[3];
            L.decode1(S.Q1.col[k], &cj, vj);
            auto it = up[ci].find({cj, vj[0] - vi[0], vj[1] - vi[1], vj[2] - vi[2]});
            double v;
            if (it != up[ci].end()) {
                v = (double)Sv[at(ci, it->second, vi)];
            } else {
                auto jt = up[cj].find({ci, vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]});
                v = jt != up[cj].end() ? (double)Sv[at(cj, jt->second, vj)] : 0.0;
            }
            qbar[k] = 0.5 * v;
        }
    }
}

template <typename real>
static int adjoint_run(ygm_ctx* ctx, int64_t nsteps, double dt, int32_t K, const uint8_t* region, double* loss,
                       double* grad) {
    const ygm::Setup& S = ctx->S;
    const ygm::Lattice& L = S.L;
    const int64_t N1 = L.N1, N2 = L.N2, T = 6LL * L.n * L.n * L.n;
    const size_t rs = sizeof(real), n1pad = (size_t)ctx->n1pad, n2pad = (size_t)ctx->pg.NP * ctx->pg.NP * ctx->pg.NP * L.c2.size();
    RegionOps R;
    build_region(ctx, region, R);
    const int nt = (int)R.tets.size();
    const int nseg = (int)((nsteps + K - 1) / K);
    // device memory of this call (freed on every exit path)
    std::vector<void*> owned;
    auto dalloc = [&](void** p, size_t bytes) -> int {
        *p = nullptr;
        if (!bytes) return 0;
        CK(cudaMalloc(p, bytes));
        owned.push_back(*p);
        CK(cudaMemsetAsync(*p, 0, bytes, ctx->stream));
        return 0;
    };
    struct Guard {
        std::vector<void*>& v;
        ~Guard() {
            for (void* p : v) cudaFree(p);
        }
    } guard{owned};
    void *ck, *seg, *ebar, *cb, *tx, *tpad, *xbp, *u, *upad, *zero2, *dump, *epad, *Sd, *lossd, *gradd;
    void *rd1, *rd2, *rep, *rim, *rgr, *rgp, *rgc, *rgv, *rmp, *rmc, *rmv, *pidx, *m1l, *m2l;
    int rc;
    const size_t q_n = S.qsym.size();
    if ((rc = dalloc(&ck, (size_t)nseg * (N1 + N2) * rs)) || (rc = dalloc(&seg, (size_t)K * (2 * N1 + N2) * rs)) ||
        (rc = dalloc(&ebar, n1pad * rs)) || (rc = dalloc(&cb, N1 * rs)) || (rc = dalloc(&tx, N1 * rs)) ||
        (rc = dalloc(&tpad, n1pad * rs)) || (rc = dalloc(&xbp, n1pad * rs)) || (rc = dalloc(&u, N2 * rs)) ||
        (rc = dalloc(&upad, n2pad * rs)) || (rc = dalloc(&zero2, N2 * rs)) || (rc = dalloc(&dump, n1pad * rs)) ||
        (rc = dalloc(&epad, n1pad * rs)) || (rc = dalloc(&Sd, q_n * rs)) || (rc = dalloc(&lossd, (size_t)nt * 8)) ||
        (rc = dalloc(&gradd, (size_t)nt * 8)))
        return rc;
    auto up = [&](void** p, const void* h, size_t bytes) -> int {
        if ((rc = dalloc(p, bytes))) return rc;
        if (bytes) CK(cudaMemcpyAsync(*p, h, bytes, cudaMemcpyHostToDevice, ctx->stream));
        return 0;
    };
    std::vector<int> pid(N1);
    for (int64_t i = 0; i < N1; ++i) {
        int c, v[3];
        L.decode1(i, &c, v);
        pid[i] = (int)(c * (long long)ctx->pg.NP * ctx->pg.NP * ctx->pg.NP +
                       ((long long)(v[2] + ctx->pg.H) * ctx->pg.NP + v[1] + ctx->pg.H) * ctx->pg.NP + v[0] + ctx->pg.H);
    }
    if ((rc = up(&rd1, R.d1.data(), R.d1.size() * 4)) || (rc = up(&rd2, R.d2.data(), R.d2.size() * 4)) ||
        (rc = up(&rep, R.epsr.data(), R.epsr.size() * 8)) || (rc = up(&rim, R.imur.data(), R.imur.size() * 8)) ||
        (rc = up(&rgr, R.g_rows.data(), R.g_rows.size() * 4)) || (rc = up(&rgp, R.g_ptr.data(), R.g_ptr.size() * 4)) ||
        (rc = up(&rgc, R.g_col.data(), R.g_col.size() * 4)) || (rc = up(&rgv, R.g_val.data(), R.g_val.size() * 8)) ||
        (rc = up(&rmp, R.m_ptr.data(), R.m_ptr.size() * 4)) || (rc = up(&rmc, R.m_col.data(), R.m_col.size() * 4)) ||
        (rc = up(&rmv, R.m_val.data(), R.m_val.size() * 8)) || (rc = up(&pidx, pid.data(), pid.size() * 4)) ||
        (rc = up(&m1l, S.M1loc.data(), S.M1loc.size() * 8)) || (rc = up(&m2l, S.M2aloc.data(), S.M2aloc.size() * 8)))
        return rc;
    // source amplitudes dt s(t_{n+1/2}) of every step (host FP64), as ygm_step computes them
    const int nsrc = ctx->nsrc;
    std::vector<double> amp((size_t)nsteps * std::max(nsrc, 1), 0.0);
    std::vector<char> on(nsteps, 0);
    for (int64_t i = 0; i < nsteps && nsrc; ++i)
        for (int q = 0; q < nsrc; ++q) {
            const ygm_source& s0 = ctx->src_cache[q];
            const double t = (i + 0.5) * dt, v = (t - s0.t0) / s0.sigma;
            const double a = dt * s0.amp * std::exp(-v * v) * std::sin(s0.omega * (t - s0.t0));
            amp[(size_t)i * nsrc + q] = a;
            if (a != 0.0) on[i] = 1;
        }
    void* ampd = nullptr;
    if (nsrc && (rc = up(&ampd, amp.data(), amp.size() * 8))) return rc;
    real* ckp = (real*)ck;
    real* sg_e = (real*)seg;
    real* sg_x = sg_e + (size_t)K * N1;
    real* sg_b = sg_x + (size_t)K * N1;
    // forward from rest (b_{-1/2} = 0: the initial half step of a zero state is zero)
    CK(cudaMemsetAsync(ctx->e, 0, N1 * rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->ep, 0, n1pad * rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[0], 0, N2 * rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[1], 0, N2 * rs, ctx->stream));
    ctx->cur = 0;
    auto fwd = [&](int64_t n, bool all, int64_t slot) {
        void* bo = ctx->b[ctx->cur];
        void* bn = ctx->b[ctx->cur ^ 1];
        if (slot >= 0) cudaMemcpyAsync(sg_e + slot * N1, ctx->e, N1 * rs, cudaMemcpyDeviceToDevice, ctx->stream);
        launch_qapply(ctx, ctx->x, all);
        launch_curl_b(ctx, ctx->x, bo, bn, dt);
        if (slot >= 0) {
            cudaMemcpyAsync(sg_x + slot * N1, ctx->x, N1 * rs, cudaMemcpyDeviceToDevice, ctx->stream);
            cudaMemcpyAsync(sg_b + slot * N2, bn, N2 * rs, cudaMemcpyDeviceToDevice, ctx->stream);
        }
        launch_curlT_e(ctx, bn, ctx->e, dt, on[n] ? (const double*)ampd + (size_t)n * nsrc : nullptr);
        ctx->cur ^= 1;
    };
    for (int64_t n = 0; n < nsteps; ++n) {
        if (n % K == 0) {
            const int64_t c = n / K;
            CK(cudaMemcpyAsync(ckp + c * (N1 + N2), ctx->e, N1 * rs, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(ckp + c * (N1 + N2) + N1, ctx->b[ctx->cur], N2 * rs, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        fwd(n, false, -1);
    }
    // reverse, one checkpoint segment at a time
    const SBlk* ball = ctx->sblks + ctx->nsblks_act;
    const size_t smem_q = (size_t)(ctx->max_ns + 8) * sizeof(int2);
    const size_t smem_e = (size_t)ctx->max_terms * sizeof(WTermL<real>);
    const int nb_all = ctx->nsblks_all;
    const dim3 gl((unsigned)std::min<int64_t>(4 * 152, (N1 + BLOCK - 1) / BLOCK)), gp((unsigned)std::min<size_t>(4 * 152, (n1pad + BLOCK - 1) / BLOCK));
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int64_t n0 = (int64_t)sgi * K, n1 = std::min<int64_t>(n0 + K, nsteps);
        CK(cudaMemcpyAsync(ctx->e, ckp + sgi * (N1 + N2), N1 * rs, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->b[ctx->cur], ckp + sgi * (N1 + N2) + N1, N2 * rs, cudaMemcpyDeviceToDevice, ctx->stream));
        launch_pad_e(ctx);
        for (int64_t n = n0; n < n1; ++n) fwd(n, true, n - n0);
        for (int64_t n = n1 - 1; n >= n0; --n) {
            const int64_t sl = n - n0;
            // cb += tau C^T M2 (C ebar)
            k_curl_b_s<real><<<ctx->nlb, SBLOCK, 0, ctx->stream>>>(ctx->lblks_b, ctx->c2, ctx->cterms, ctx->pg, ctx->sg.NX,
                                                                   (const real*)ebar, (const real*)zero2, (real*)u,
                                                                   (real*)upad, split_tau<real>(-1.0));
            k_curlT_e_s<real><<<ctx->nle, SBLOCK, smem_e, ctx->stream>>>(ctx->lblks_e, ctx->c1, ctx->pbeg,
                                                                        (const WTermL<real>*)ctx->wterms, ctx->pg, ctx->sg.NX,
                                                                        (const real*)upad, (real*)cb, split_tau<real>(dt),
                                                                        (real*)dump, nullptr, nullptr, nullptr);
            // cb += tau C^T M2^R b_{n+1/2}
            const int ngr = (int)R.g_rows.size();
            if (ngr)
                k_csr_add<real><<<(ngr + 255) / 256, 256, 0, ctx->stream>>>(ngr, (const int*)rgr, (const int*)rgp, (const int*)rgc,
                                                                            (const double*)rgv, sg_b + sl * N2, (real*)cb, dt);
            // xbar = -tau cb + tau M1^R x_n ; ebar += Q1 xbar
            k_xbar<real><<<gl, BLOCK, 0, ctx->stream>>>(N1, (const int*)pidx, (const int*)rmp, (const int*)rmc, (const double*)rmv,
                                                        (const real*)cb, sg_x + sl * N1, dt, (real*)xbp);
            k_qapply_s<real, false><<<nb_all, SBLOCK, smem_q, ctx->stream>>>(ball, ctx->c1, ctx->soff2, ctx->sg,
                                                                             (const real*)ctx->qsd, (const real*)xbp, (real*)tx,
                                                                             (real*)tpad, nullptr);
            k_pad_add<real><<<gp, BLOCK, 0, ctx->stream>>>((long long)n1pad, (real*)ebar, (const real*)tpad);
            // Q1bar += xbar e_n^T (stored pairs), and the region terms of step n
            k_pad_e<real><<<ctx->nplanes, BLOCK, 0, ctx->stream>>>(ctx->c1, ctx->planes, ctx->pg, 0, sg_e + sl * N1, (real*)epad);
            k_q1bar<real><<<nb_all, SBLOCK, smem_q, ctx->stream>>>(ball, ctx->c1, ctx->soff2, ctx->sg, (const real*)xbp,
                                                                    (const real*)epad, (real*)Sd);
            if (nt)
                k_region<real><<<(nt + 127) / 128, 128, 0, ctx->stream>>>(nt, L.n1, L.n2a, (const int*)rd1, (const int*)rd2,
                                                                          (const double*)m1l, (const double*)m2l,
                                                                          (const double*)rep, (const double*)rim,
                                                                          sg_x + sl * N1, sg_b + sl * N2, dt,
                                                                          (double*)lossd, (double*)gradd);
            ctx->launches += 9;
        }
        CK(cudaGetLastError());
    }
    std::vector<real> Sh(q_n);
    std::vector<double> lh(nt), gh(nt);
    CK(cudaMemcpyAsync(Sh.data(), Sd, q_n * rs, cudaMemcpyDeviceToHost, ctx->stream));
    if (nt) {
        CK(cudaMemcpyAsync(lh.data(), lossd, (size_t)nt * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(gh.data(), gradd, (size_t)nt * 8, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    // the context's state is left at rest
    CK(cudaMemsetAsync(ctx->e, 0, N1 * rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->ep, 0, n1pad * rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[0], 0, N2 * rs, ctx->stream));
    CK(cudaMemsetAsync(ctx->b[1], 0, N2 * rs, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->cur = 0;
    ctx->staggered = false;
    ctx->step = ctx->step_base = 0;
    ctx->t_base = 0.0;
    ctx->hist_n = 0;
    double Ls = 0.0;
    for (int i = 0; i < nt; ++i) Ls += lh[i];
    *loss = Ls;
    if (grad) {
        std::vector<double> qbar;
        pairs_to_csr(S, Sh, qbar);
        if ((rc = ygm::q1_vjp(ctx->S, qbar.data(), grad, 0)))
            return fail(ctx, rc == -1 ? YGM_EINVAL : YGM_ENOTSPD, "adjoint: the SPAI derivative failed");
        for (int i = 0; i < nt; ++i) grad[R.tets[i]] += gh[i];
    }
    (void)T;
    return YGM_OK;
}

extern "C" {

int ygm_adjoint(ygm_ctx* ctx, int64_t nsteps, double dt, const ygm_source* src, int32_t n_src, const uint8_t* region,
                int32_t checkpoint_every, double* loss, double* grad_eps) {
    if (ctx && ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (!ctx || !region || !loss) return fail(ctx, YGM_EINVAL, "NULL argument");
    if (nsteps < 1 || !(dt > 0) || !std::isfinite(dt) || checkpoint_every < 1)
        return fail(ctx, YGM_EINVAL, "need nsteps >= 1, finite dt > 0 and checkpoint_every >= 1");
    if (dt > ctx->S.tau_cfl * (1.0 + 1e-12))
        return fail(ctx, YGM_ECFL, "dt exceeds the CFL bound 2/omega_max (Prop. stability)");
    if (!ctx->use_sym || ctx->n_rhs != 1 || !ctx->wterms || ctx->split_w.size() != 1)
        return fail(ctx, YGM_EINVAL, "ygm_adjoint needs a one-column Strang context with uniform mu on the lattice path");
    if (n_src < 0 || (n_src > 0 && !src)) return fail(ctx, YGM_EINVAL, "bad source list");
    int rc = set_sources(ctx, src, n_src);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    const int32_t K = (int32_t)std::min<int64_t>(checkpoint_every, nsteps);
    return ctx->precision == YGM_FP64 ? adjoint_run<double>(ctx, nsteps, dt, K, region, loss, grad_eps)
                                      : adjoint_run<float>(ctx, nsteps, dt, K, region, loss, grad_eps);
}

int ygm_qapply_counts(const ygm_ctx* ctx, int all_rows, int64_t* rows, int64_t* unique_values,
                      int64_t* stored_values) {
    if (!ctx) return YGM_EINVAL;
    if (ctx->host_only) return YGM_ENODEV;
    const int a = all_rows ? 1 : 0;
    if (rows) *rows = ctx->qc_rows[a];
    if (unique_values) *unique_values = ctx->qc_unique[a];
    if (stored_values) *stored_values = ctx->qc_stored[a];
    return YGM_OK;
}

int ygm_q1_info(const ygm_ctx* ctx, double* lmin, double* lmax, double* shift, double* omega_max_sq,
                int32_t* pattern, int32_t* ortho) {
    if (!ctx) return YGM_EINVAL;
    if (lmin) *lmin = ctx->S.lmin;
    if (lmax) *lmax = ctx->S.lmax;
    if (shift) *shift = ctx->S.shift;
    if (omega_max_sq) *omega_max_sq = ctx->S.omega_max_sq;
    if (pattern) *pattern = ctx->S.q1_pattern;
    if (ortho) *ortho = ctx->S.ortho ? 1 : 0;
    return YGM_OK;
}

int ygm_local_blocks(const ygm_ctx* ctx, int32_t* n1, int32_t* n2a, double* M1, double* M2a) {
    if (!ctx) return YGM_EINVAL;
    if (n1) *n1 = ctx->S.L.n1;
    if (n2a) *n2a = ctx->S.L.n2a;
    if (M1) std::copy(ctx->S.M1loc.begin(), ctx->S.M1loc.end(), M1);
    if (M2a) std::copy(ctx->S.M2aloc.begin(), ctx->S.M2aloc.end(), M2a);
    return YGM_OK;
}

int ygm_set_qapply(ygm_ctx* ctx, int32_t kernel, int32_t stages, int32_t* blocks_per_sm) {
    if (!ctx) return YGM_EINVAL;
    if (ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (kernel < 0 || kernel > 2) return fail(ctx, YGM_EINVAL, "kernel must be 0 (automatic), 1 (k_qapply_s) or 2 (k_qapply_t)");
    if (!ctx->use_sym) return fail(ctx, YGM_EINVAL, "no upper-triangle Q1 path on this context (n_rhs > 1)");
    if (kernel == 2 && !ctx->qt_ok) return fail(ctx, YGM_EINVAL, "k_qapply_t is not available on this context");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    int bps = 0;
    if (ctx->qt_ok) {
        const int rc = qt_configure(ctx, stages, &bps);
        if (rc) return rc;
    } else if (stages) {
        return fail(ctx, YGM_EINVAL, "stages apply to k_qapply_t only");
    }
    ctx->qt_mode = kernel;
    if (blocks_per_sm) {
        if (!ctx->qt_ok || kernel != 2) {
            const size_t smem = (size_t)(ctx->max_ns + 8) * sizeof(int2);
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &bps, ctx->precision == YGM_FP64 ? (const void*)k_qapply_s<double, false> : (const void*)k_qapply_s<float, false>,
                SBLOCK, smem));
        }
        *blocks_per_sm = bps;
    }
    return YGM_OK;
}

int ygm_set_launch(ygm_ctx* ctx, int32_t pdl) {
    if (!ctx) return YGM_EINVAL;
    if (ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    if (pdl != 0 && pdl != 1) return fail(ctx, YGM_EINVAL, "pdl must be 0 or 1");
    ctx->pdl = pdl != 0;
    return YGM_OK;
}

int ygm_kernel_timing(ygm_ctx* ctx, int enable) {
    if (!ctx) return YGM_EINVAL;
    if (ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    ctx->timing = enable != 0;
    return YGM_OK;
}

int ygm_kernel_times(ygm_ctx* ctx, double* ms, int64_t* count) {
    if (!ctx || !ms || !count) return fail(ctx, YGM_EINVAL, "NULL argument");
    if (ctx->host_only) return fail(ctx, YGM_ENODEV, "context was created host-only (device = -1)");
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < NKIND; ++i) {
        ms[i] = 0.0;
        count[i] = 0;
    }
    for (auto& [kind, i0] : ctx->ev_rec) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ctx->ev_pool[i0], ctx->ev_pool[i0 + 1]));
        ms[kind] += t;
        count[kind] += 1;
    }
    ctx->ev_rec.clear();
    ctx->ev_used = 0;
    return YGM_OK;
}

int ygm_launch_count(const ygm_ctx* ctx, int64_t* count) {
    if (!ctx || !count) return YGM_EINVAL;
    *count = ctx->launches;
    return YGM_OK;
}

void ygm_destroy(ygm_ctx* ctx) {
    if (!ctx) return;
    if (ctx->host_only) {
        delete ctx;
        return;
    }
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    void* ptrs[] = {ctx->e,     ctx->b[0],  ctx->b[1], ctx->x,     ctx->bscr,  ctx->q,     ctx->W,     ctx->inv_mu,
                    ctx->sw,    ctx->M2a,   ctx->c1,   ctx->c2,    ctx->slots, ctx->terms, ctx->inc,   ctx->loc2,
                    ctx->rowsE, ctx->part, ctx->hist,  ctx->dsrc,  ctx->sdofs, ctx->ep,   ctx->qf,    ctx->pblks,
                    ctx->soff,  ctx->planes, ctx->spdofs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
    for (int i = 0; i < 2; ++i) {
        if (ctx->damp_ev[i]) cudaEventDestroy(ctx->damp_ev[i]);
        if (ctx->damp[i]) cudaFree(ctx->damp[i]);
        if (ctx->hamp[i]) cudaFreeHost(ctx->hamp[i]);
    }
    void* more[] = {ctx->qslots, ctx->qblocks, ctx->eblocks, ctx->bblocks, ctx->pterms, ctx->pbeg,
                    ctx->qsd,    ctx->soff2,   ctx->sblks,   ctx->xp,      ctx->bp,     ctx->wterms,
                    ctx->cterms, ctx->lblks_b, ctx->lblks_e, ctx->qpart,  ctx->ticket, ctx->M2af,
                    ctx->lblks_es, ctx->sbeg,    ctx->sent,     ctx->uterm,  ctx->acls,  ctx->wt,
                    ctx->dev_err};
    for (void* p : more)
        if (p) cudaFree(p);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
