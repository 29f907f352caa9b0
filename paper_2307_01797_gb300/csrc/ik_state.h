// ik_state.h -- device state of one itokmc handle and the host-side launchers
// shared by the translation units of libitokmc.
#pragma once
#include <cstddef>
#include <atomic>
#include <cstdint>
#include <cmath>
#include <cuda_runtime.h>

#include "ik_common.cuh"

namespace ik {

// FP64-form particle record: absolute position, global cell (r n^3 + c),
// weight (physical electrons).  32 bytes, loaded as two 16-byte vectors.
struct alignas(16) P64 {
    double x, y, z;
    uint32_t cell;
    uint32_t w;
};

// Mixed-form particle record: position inside the cell in cell units
// [0, 1), weight.  16 bytes; the global cell lives in a separate array.
struct alignas(16) P32 {
    float ox, oy, oz;
    uint32_t w;
};

// Cell-centred field: E components and |E| = sqrt((Ex^2 + Ey^2) + Ez^2).
struct alignas(16) E64 {
    double x, y, z, m;
};

struct Mover {       // a particle that changed cell in the push
    uint32_t g;      // new global cell
    uint32_t i;      // index in the pre-push array
};

struct Photo {       // an absorbed superphoton (photoelectron)
    double x, y, z;  // absorption point (FP64 form) / cell offsets (mixed)
    uint32_t g;      // global absorption cell
    uint32_t src;    // source cell within the realization
    uint32_t slot;   // superphoton slot in the source cell
    uint32_t w;      // weight
};

// Flags in the push key word.
constexpr uint32_t KEY_DEAD = 0x80000000u;
constexpr uint32_t KEY_MOVER = 0x40000000u;
constexpr uint32_t KEY_MASK = 0x3fffffffu;

constexpr int TPB = 256;        // threads per block of the particle passes
constexpr int MAX_R = 1024;     // realizations per handle

// Device counters of one step (zeroed at the start of each stage).
struct Counters {
    unsigned long long n_movers;
    unsigned long long n_photo;
    unsigned long long n_new;          // product + photo particles
    unsigned long long ion, att, phot; // firings
    unsigned long long rec_ep, rec_np; // recombination firings
    unsigned long long absorbed_w;
    unsigned long long photo_slots;    // sum over cells of min(N_gamma, N_new)
    unsigned int n_photo_cells;        // photon-emitting cells listed by the KMC
    unsigned int n_kmc_cells;          // cells with X_e > 0 listed for the KMC
    unsigned long long merge_cells, merge_elems, merge_elems2, merge_maxm;   // merge workload
    unsigned long long rho_absmax;     // max |rho_fixed| of the last deposit
    unsigned int err;                  // DERR_* bits
    unsigned int kmc_fail_cell;
    unsigned long long outflow[MAX_R];
    unsigned long long lost[MAX_R];
};

// Variable-coefficient operator of one level (semi-implicit field): the cell
// coefficient c, the coefficients of the +x, +y, +z faces of each cell (0
// where the face is on the boundary), the diagonal and its inverse.
struct VCLevel {
    double* c = nullptr;
    double* fx = nullptr;  double* fy = nullptr;  double* fz = nullptr;
    double* dg = nullptr;  double* idg = nullptr;
};

struct MGLevel {
    int n;                 // cells per axis on this level
    double h;              // cell size
    double* phi;  double* rhs;  double* res;   // FP64 (size R n^3)
    float* phi32; float* rhs32;                 // FP32 inner V-cycles
};

constexpr int MAX_LEVELS = 12;

struct Dev {
    // particles (ping-pong)
    P64* recA = nullptr;  P64* recB = nullptr;
    P32* rA32 = nullptr;  P32* rB32 = nullptr;
    uint32_t* cellA32 = nullptr;  uint32_t* cellB32 = nullptr;
    uint32_t* keyB = nullptr;
    uint32_t* cell_start = nullptr;     // G + 1, current array
    uint32_t* cell_start_B = nullptr;   // G + 1, scratch
    // per-cell transport counters
    int32_t* cnt_new = nullptr;  int32_t* in_cnt = nullptr;  int32_t* in_before = nullptr;
    int32_t* cursor = nullptr;   int64_t* delta = nullptr;   uint32_t* in_off = nullptr;
    uint32_t* blk_stay = nullptr;  uint32_t* blk_prefix = nullptr;
    Mover* movers = nullptr;  uint32_t* mover_sorted = nullptr;
    // mesh
    unsigned long long* ne_fix = nullptr;  unsigned long long* Xe = nullptr;
    int64_t* Npos = nullptr;  int64_t* Nneg = nullptr;  int64_t* rho = nullptr;
    E64* E = nullptr;  float4* E32 = nullptr;
    // chemistry
    int64_t* fired = nullptr;          // 5 G: ionizations, attachments, photons, e-ion and ion-ion
                                       // recombinations of the last KMC
    int64_t* gain = nullptr;           // Gp: net gain of each particle cell's species in the last KMC
    uint32_t* step_dev = nullptr;      // the step counter of graph-replayed steps
    // photons
    Photo* photos = nullptr;  uint32_t* photo_sorted = nullptr;
    int32_t* photo_cnt = nullptr;  int32_t* photo_cursor = nullptr;
    unsigned long long* photo_w = nullptr;  uint32_t* photo_off = nullptr;
    // merge
    uint32_t* out_start = nullptr;     // G + 1
    uint64_t* work_off = nullptr;      // G + 1
    uint32_t* small_list = nullptr;    // G: non-empty cells of merge tier 0 (small shared scratch)
    uint32_t* mid_list = nullptr;      // G: ... tier 1 (large shared scratch)
    uint32_t* big_list = nullptr;      // G: ... tier 2 (scratch in the work area)
    uint32_t* list_n = nullptr;        // 2 counts
    uint32_t* pc_list = nullptr;       // G: photon-emitting cells
    unsigned char* work = nullptr;  size_t work_bytes = 0;   // merge scratch of tier-2 cells
    // scans
    long long* scan_blk = nullptr;  size_t scan_blk_elems = 0;
    // multigrid
    MGLevel lev[MAX_LEVELS];
    int nlev = 0;
    double* norm_part = nullptr;  double* norm_out = nullptr;  size_t norm_blocks = 0;
    double* norm_host = nullptr;       // 2 R doubles (pinned or stack) for the norm readback
    // counters
    Counters* ctr = nullptr;
    Counters* ctr_host = nullptr;      // pinned mirror
    uint32_t* sort_tmp = nullptr;      // radix-sort scratch (4 x capacity u32)
    uint32_t mover_cap = 0, photo_cap = 0;
    uint64_t work_cap = 0;             // merge work area, 32-byte units
    double* stage = nullptr;           // 3 G doubles: field upload/readback
    // CUDA graphs of the correction sweep (FP32: zero + two V-cycles) and of
    // one FP64 V-cycle, captured once per smoother pair and replayed
    cudaGraphExec_t vgraph[3] = { nullptr, nullptr, nullptr };
    int vgraph_nu[3][2] = { { 0, 0 }, { 0, 0 }, { 0, 0 } };
    unsigned long long vgraph_kernels[3] = { 0, 0, 0 };
    VCLevel vc[MAX_LEVELS];            // semi-implicit operator per level (allocated on first use)
    bool direct_cycles = false;        // launch the cycles directly (no capture)
    cudaStream_t side = nullptr;       // merge tiers 1 and 2 run beside tier 0
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    E64* E_next = nullptr;             // field of the next step, solved while the
    float4* E32_next = nullptr;        //   particle stages of this step still run
    bool mixed = false;                // FP32 particle form
    int phi_F = 0;                     // potential in int64 units of 2^-phi_F V (0: FP64 potential)
    void* phi_prev = nullptr;          // potential of the previous solve (initial-guess extrapolation)
    bool have_prev = false;
};

// Right-hand side constants: b = -rho_fixed qscale, minus bc_top in the top
// layer (electrode ghost 2 phi_b - phi_1).
inline void rhs_consts(const Params& P, double& qscale, double& bc_top)
{
    const double dV = P.h[0] * P.h[1] * P.h[2];
    qscale = 1.602176634e-19 * std::ldexp(1.0, -3 * P.frac_bits) / dV / 8.8541878128e-12;
    const double phi_top = P.E0 * (P.hi[2] - P.lo[2]);
    bc_top = 2.0 * phi_top / (P.h[2] * P.h[2]);
}

// Fixed-point bits F of the potential for a bound |phi| <= phi_max: keeps
// |Phi| = |phi| 2^F at most 2^58, so sums of eight stay inside int64.
inline int phi_fixed_bits(double phi_max)
{
    int e = 0;
    std::frexp(phi_max > 1.0 ? phi_max : 1.0, &e);   // phi_max < 2^e
    const int F = 58 - e;
    return F < 8 ? 8 : (F > 52 ? 52 : F);
}

// Bound on |phi| of the discrete solution: the electrode potential plus the
// 1D Dirichlet bound max|b| Lz^2 / 8 of the space charge, doubled for the
// iterates.
inline double phi_bound(const Params& P, unsigned long long rho_absmax)
{
    double qscale, bc_top;
    rhs_consts(P, qscale, bc_top);
    const double Lz = P.hi[2] - P.lo[2];
    return 2.0 * (std::fabs(P.E0 * Lz) + (double)rho_absmax * qscale * Lz * Lz / 8.0) + 1.0;
}

// ------------------------------------------------------------- launchers
// ik_particles.cu
void launch_transport(const Params& P, Dev& d, uint32_t N, cudaStream_t s, const uint32_t* Ndev = nullptr);
void field_solve_fixed(const Params& P, Dev& d, int precision, int nu1, int nu2, int cycles, cudaStream_t s);
void lower_phi_scale(const Params& P, Dev& d, int F, cudaStream_t s);
float time_push(const Params& P, Dev& d, uint32_t N, cudaStream_t s, int reps);
void launch_diff_flag(const unsigned long long* a, const unsigned long long* b, uint64_t n, unsigned int* flag,
                      cudaStream_t s);
void launch_transport_finish(const Params& P, Dev& d, uint32_t N, uint64_t G, cudaStream_t s,
                             const uint32_t* Ndev = nullptr);
void launch_deposit_only(const Params& P, Dev& d, uint32_t N, cudaStream_t s);
void launch_rho(const Params& P, Dev& d, uint64_t G, cudaStream_t s);
void launch_zig_init(cudaStream_t s);
void launch_kmc(const Params& P, Dev& d, uint64_t G, cudaStream_t s);
void launch_step_maxima(const Params& P, Dev& d, unsigned long long* m, cudaStream_t s);
void launch_kmc0d(const Params& P, bool mixed, double Em, long long X0, uint32_t nreal, int nsteps, long long* X,
                  Counters* ctr, cudaStream_t s);
void launch_particles_a(const Params& P, Dev& d, uint64_t G, cudaStream_t s);
void launch_particles_b(const Params& P, Dev& d, uint64_t G, cudaStream_t s);
void launch_diffuse(const Params& P, Dev& d, uint32_t N, cudaStream_t s);
void launch_deposit_B(const Params& P, Dev& d, uint32_t N, cudaStream_t s);
void launch_advect(const Params& P, Dev& d, uint32_t N, cudaStream_t s);
// ik_sort.cu
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                      uint32_t n, int key_bits, cudaStream_t s, long long* blk_scratch,
                      size_t blk_scratch_elems);
size_t radix_scratch_elems(uint32_t cap);
void launch_set_particles(const Params& P, Dev& d, const double* x, const double* y,
                          const double* z, const uint32_t* w, const int32_t* real, const int32_t* species,
                          uint32_t n, uint64_t G, cudaStream_t s);
// ik_field.cu
int field_solve(const Params& P, Dev& d, int precision, double rtol, int nu1, int nu2, unsigned long long rho_absmax,
                int max_cycles, cudaStream_t s, int* cycles_out, double* rel_out, bool extrapolate = false);
void launch_efield(const Params& P, Dev& d, cudaStream_t s);
void launch_efield_to(const Params& P, Dev& d, cudaStream_t s, E64* E, float4* E32);
void launch_semi_coef(const Params& P, Dev& d, double* c0, cudaStream_t s);
int field_solve_vc(const Params& P, Dev& d, double* acc, double* acc_host, double rtol, int nu1, int nu2,
                   int max_cycles, cudaStream_t s, int* cycles_out, double* rel_out);
void launch_phi_to_double(const Params& P, Dev& d, double* out, cudaStream_t s);
void launch_pack_field(const Params& P, Dev& d, const double* E3, cudaStream_t s);
void launch_unpack_field(const Params& P, Dev& d, double* E3, cudaStream_t s);

// Kernel launches issued by this library (all handles), for the benchmark's
// launch count.
extern std::atomic<unsigned long long> g_launches;

// Last error of a call made without a handle (itokmc_last_error(NULL)).
extern thread_local char g_noh_err[256];
void set_global_error(const char* msg);

// generic 3-phase exclusive scan over G cells with C channels (ik_particles.cu)
size_t scan_scratch_elems(uint64_t G, int C);

}  // namespace ik
