// Host-side FP64 set-up of the GYM operators on the Kuhn-split PEC cube.
//
// Everything here runs once per context: lattice classes and stencils, order-k local
// bases, exact element integrals, M1(eps), M2(mu), the integer curl, the SPAI Q1
// (Sec. 5, Eq. NormalEqSolve) and the CFL bound (Prop. stability).  On request it also
// computes the operator-probed SPAI (Sec. 5.1), the cavity modes used as its probes, and the
// derivative of the SPAI with respect to the per-tet permittivity.  The device kernels only
// ever see the packed tables produced at the end.
#pragma once
#include <array>
#include <map>
#include <cstdint>
#include <string>
#include <vector>

namespace ygm {

// ---------------------------------------------------------------- lattice / numbering
struct Box {
    int lo[3];
    int num[3];
    int64_t offset;  // first global index of the class
    int64_t size;    // num[0] * num[1] * num[2]
};

struct DofClass {
    int kind;     // 0 edge, 1 face, 2 tet
    int shape;    // shape index inside the kind
    int j;        // DoF index inside the entity
    int ext;      // extent bit mask (union of the entity's vertex offsets)
    bool active;  // 1-forms: carries curl (not a gradient); 2-forms: a row of C
    Box box;
};

// A local DoF of a tet of a given shape: its class and the lattice offset (0/1 per axis)
// of the entity anchor relative to the tet's cube.
struct LocalDof {
    int cls;
    int off[3];
};

// A tet incident to an entity: cube offset (relative to the entity anchor), tet shape,
// local index of the DoF in that tet.
struct Incidence {
    int dcube[3];
    int shape;
    int loc;
};

// A neighbour DoF in a stencil: class and anchor offset.
struct Nbr {
    int cls;
    int d[3];
    bool operator<(const Nbr& o) const;
    bool operator==(const Nbr& o) const;
};

struct Lattice {
    int n = 0, k = 0;
    double h = 0;
    std::vector<DofClass> c1, c2;   // 1-form and 2-form classes
    int64_t N1 = 0, N2 = 0;
    int n1 = 0, n2 = 0, n2a = 0;    // local DoFs per tet (n2a = curl-carrying 2-forms)
    std::vector<LocalDof> loc1[6], loc2[6];   // local order of every tet shape
    std::vector<int> act2;          // local 2-form indices that are rows of C (size n2a)
    std::vector<std::vector<Incidence>> inc1;  // per 1-form class: incident tets

    void build(int n, int k, double side);
    int64_t index(const std::vector<DofClass>& cls, int c, int x, int y, int z) const;
    int64_t index1(int c, int x, int y, int z) const { return index(c1, c, x, y, z); }
    int64_t index2(int c, int x, int y, int z) const { return index(c2, c, x, y, z); }
    // global DoFs of tet t (-1 where PEC removed them)
    void tet_dofs1(int64_t t, int64_t* out) const;
    void tet_dofs2(int64_t t, int64_t* out) const;
    // (class, anchor) of a global 1-form index
    void decode1(int64_t g, int* cls, int v[3]) const;
};

// ---------------------------------------------------------------- sparse matrices
struct Csr {
    int64_t nrows = 0, ncols = 0;
    std::vector<int64_t> ptr;
    std::vector<int64_t> col;
    std::vector<double> val;
    double get(int64_t i, int64_t j) const;   // 0 if absent
    void matvec(const double* x, double* y, int threads) const;
    void matvec_t(const double* x, double* y) const;  // y = A^T x (serial)
};

Csr transpose(const Csr& A);
Csr spgemm(const Csr& A, const Csr& B, int threads);

// ---------------------------------------------------------------- set-up result
struct Setup {
    Lattice L;
    std::vector<double> eps, mu;                 // per tet
    std::vector<double> M1loc, M2aloc;           // n1 x n1, n2a x n2a
    std::vector<double> Wloc;                    // n1 x n2a : C_loc^T M2a_loc
    std::vector<int> Cloc;                       // n2a x n1 integer local curl (active rows)
    Csr M1, Q1;                                  // global FP64
    double lmin = 0, lmax = 0, shift = 0;        // SPD check of Q1
    double omega_max_sq = 0, tau_cfl = 0;
    int q1_pattern = 0;
    bool ortho = false;
    std::string err;

    // device-facing tables ---------------------------------------------------
    // Q1 stencil: for each 1-form class c, upper slots (stored in row c) and lower slots
    // (read from the neighbour's upper slot).  Entry encoding in StencilSlot.
    struct StencilSlot {
        int32_t cls;      // neighbour class
        int8_t d[3];      // neighbour anchor offset
        int8_t upper;     // 1: value stored in this row's slot `slot`; 0: in neighbour's slot `slot`
        int32_t slot;     // slot index inside the owning row's upper list
    };
    std::vector<int32_t> st_begin;               // per class, into st_slots (size C1 + 1)
    std::vector<StencilSlot> st_slots;
    std::vector<int32_t> n_upper;                // per class
    std::vector<int64_t> qoff;                   // per class: offset of its (slot-major) value block
    std::vector<double> qvals;                   // packed upper values, [class][slot][box index]
    // full row storage for the streamed Q1 apply: every slot of the class stencil (upper and
    // lower) for every row, [class][slot][z-plane padded to 4 entries][y][x]
    std::vector<int64_t> qf_off;                 // per class: first entry
    std::vector<int64_t> qf_plane;               // per class: padded plane length (multiple of 4)
    std::vector<double> qfull;
    // upper-triangle storage on the common anchor lattice for the plane-sweep Q1 apply: every
    // class and upper slot owns an NZ x NY x NX box indexed by the row's absolute anchor
    // (qsym[qs_base[c] + s * qs_vol + (vz * NY + vy) * NX + vx]), zero where no row exists, with a
    // zeroed guard of qs_guard entries (at least 512) at both ends so every stencil neighbour
    // address, and every 256-point run the kernels copy from one, is in range
    int qs_nx = 0, qs_ny = 0, qs_nz = 0, qs_h = 0;
    int64_t qs_vol = 0, qs_guard = 0;
    std::vector<int64_t> qs_base;                // per class (size C1 + 1; the last is the end of the data)
    std::vector<double> qsym;
};

// Fill qfull from Q1 and the stencil tables (called by build_setup and install_q1).
void pack_full(Setup& S, int threads);
// Fill qsym from qvals (called after pack_full).  Returns false if an anchor lies outside [0, n).
bool pack_sym(Setup& S, int threads);

int build_setup(Setup& S, int n, double side, int k, const double* eps, const double* mu,
                int q1_pattern, int threads);

// Replace Q1 by a caller's symmetric matrix on this context's stencil pattern, repack the
// device-facing values and recompute the SPD check and the CFL bound.
int install_q1(Setup& S, const int64_t* rowptr, const int64_t* colind, const double* val, int threads);
int refresh_spectrum(Setup& S, int threads);
// Repack qvals / qfull / qsym from S.Q1 and refresh the SPD check and CFL bound.
int repack_q1(Setup& S, int threads);
// Operator-probed SPAI (Sec. 5.1) on the pattern of the current Q1, warm-started from it.
// V: N1 x np probe modes (column-major).  Returns 0, -1 (bad input), -2 (PCG not converged,
// Q1 unchanged), -3 (not SPD after the update).
int spai_op(Setup& S, const double* V, int np, double lam, int maxit, double tol, int threads, int* iters,
            double* relres);
// Lowest `count` non-kernel eigenpairs of P2 v = lambda M1 v (v^T M1 v = 1), V column-major N1 x count.
// Returns 0, -1 (bad input), -2 (not converged), -3 (internal / inner solve failure).
int cavity_modes(Setup& S, int count, double* V, double* lam, int maxit, double tol, int threads, int* iters);
// dL/d eps (per tet, length 6 n^3) through Q1 for q1bar = dL/dQ1 on the Q1 CSR pattern: the column
// SPAI (order 1) or the entity-orthonormal SPAI (orders >= 2).  Returns 0, -1 (asymmetric
// pattern), -3 (a normal matrix not SPD).
int q1_vjp(Setup& S, const double* q1bar, double* grad, int threads);

// Source vector of one dipole: tet index and the n1 weights d . Lambda1_i(x0) (global DoFs).
int dipole_weights(const Setup& S, const double x[3], const double d[3], std::vector<int64_t>& dofs,
                   std::vector<double>& w);

// e0 = M1 Pi E0 (k = 1 canonical interpolant, k >= 2 L2 load vector)
int project_E(const Setup& S, void (*E0)(const double*, double*, void*), void* user,
              std::vector<double>& e0, int threads);

}  // namespace ygm
