// ik_api.cu -- the C ABI of libitokmc (declared in include/itokmc.h): handle
// life cycle, device memory, state upload/readback and the step driver.
#include <algorithm>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/itokmc.h"
#include "ik_common.cuh"
#include "ik_state.h"
#include "ik_handle.h"

namespace ik {
std::atomic<unsigned long long> g_launches{0};

// Message of the last error raised without a handle (fixed storage: no
// allocation on this path).
thread_local char g_noh_err[256] = "";
void set_global_error(const char* msg)
{
    snprintf(g_noh_err, sizeof g_noh_err, "%s", msg);
}
}

struct itokmc_handle {
    itokmc_config cfg;
    ik::Params P;
    ik::Dev d;
    cudaStream_t s = nullptr;
    cudaStream_t sf = nullptr;    // field stream (the solve overlaps the particle stages)
    cudaEvent_t fork = nullptr, join = nullptr;
    int device = 0;
    uint64_t G = 0;           // cells of all realizations (field, KMC)
    uint64_t Gp = 0;          // particle cells: G per species block (S G)
    // graph-replayed steps: capture stream, cached graphs keyed by the device
    // state they start from, the cycle count of their field solve, and the
    // last step's buffer use (the headroom a replay needs)
    cudaStream_t scap = nullptr;
    struct GraphEntry;
    std::vector<GraphEntry*> graphs;
    int graph_cycles = 0;
    uint32_t graph_nbound = 0;  // particle-count bound the next replay's grids cover
    uint64_t last_photo_slots = 0, last_work = 0;
    unsigned long long last_rho_absmax = 0;
    int steps_done = 0;
    uint32_t N = 0;           // particle count (host copy)
    uint32_t cap = 0;
    int64_t step = 0;
    int field_prec = 0;
    int stage = 0;                // stage order, see checked_stage
    bool poisoned = false;
    std::string err;
    std::mutex emtx;              // err/poisoned are written by the step and field threads
    std::vector<void*> allocs;
    itokmc_stats st{};
    cudaEvent_t ev[8]{};
    struct Readback { uint32_t N; uint32_t step; uint64_t work_need; ik::Counters ctr; }* rb = nullptr;  // pinned
};

namespace {


int fail(itokmc_handle* h, int code, const std::string& msg)
{
    if (h) {
        std::lock_guard<std::mutex> lk(h->emtx);
        h->err = msg;
        if (code == ITOKMC_ERR_CUDA || code == ITOKMC_ERR_TIMEOUT) h->poisoned = true;
    } else {
        ik::set_global_error(msg.c_str());
    }
    return code;
}

int cuda_check(itokmc_handle* h, cudaError_t e, const char* where)
{
    if (e == cudaSuccess) return ITOKMC_OK;
    return fail(h, ITOKMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define IK_CHECK(h, call)                                        \
    do {                                                         \
        int _rc = cuda_check((h), (call), #call);                \
        if (_rc) return _rc;                                     \
    } while (0)

#define IK_GUARD(h)                                              \
    do {                                                         \
        if (!(h)) return ITOKMC_ERR_ARG;                         \
        if ((h)->poisoned) return ITOKMC_ERR_POISONED;           \
    } while (0)

void* dalloc(itokmc_handle* h, size_t bytes, int* rc)
{
    if (*rc) return nullptr;
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (h->cfg.alloc) {
        p = h->cfg.alloc(bytes, h->cfg.alloc_ctx);
        if (!p) { *rc = fail(h, ITOKMC_ERR_OOM, "allocator returned NULL"); return nullptr; }
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, h->s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *rc = fail(h, ITOKMC_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
            return nullptr;
        }
    }
    h->allocs.push_back(p);
    if (cudaMemsetAsync(p, 0, bytes, h->s) != cudaSuccess) *rc = fail(h, ITOKMC_ERR_CUDA, "memset");
    return p;
}

template <class T>
T* dalloc_n(itokmc_handle* h, size_t n, int* rc) { return reinterpret_cast<T*>(dalloc(h, n * sizeof(T), rc)); }

void dfree(itokmc_handle* h, void* p)
{
    if (!p) return;
    for (size_t i = 0; i < h->allocs.size(); ++i)
        if (h->allocs[i] == p) { h->allocs.erase(h->allocs.begin() + i); break; }
    if (h->cfg.free_fn) h->cfg.free_fn(p, h->cfg.alloc_ctx);
    else cudaFreeAsync(p, h->s);
}

// Grows the photon list to hold at least `need` superphotons (geometric).
int ensure_photo_cap(itokmc_handle* h, uint64_t need)
{
    if (need <= h->d.photo_cap) return ITOKMC_OK;
    if (need > 0xfff00000ull) return ITOKMC_ERR_CAPACITY;
    uint64_t cap = std::max<uint64_t>(need + need / 4, 2ull * h->d.photo_cap);
    if (cap > 0xfff00000ull) cap = 0xfff00000ull;
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    dfree(h, h->d.photos);
    dfree(h, h->d.photo_sorted);
    int rc = 0;
    h->d.photos = dalloc_n<ik::Photo>(h, cap, &rc);
    h->d.photo_sorted = dalloc_n<uint32_t>(h, cap, &rc);
    if (rc) return rc;
    h->d.photo_cap = (uint32_t)cap;
    return ITOKMC_OK;
}

// Merge work area of `cap` 32-byte units.
void set_work(itokmc_handle* h, unsigned char* p, uint64_t cap)
{
    h->d.work = p;
    h->d.work_cap = cap;
    h->d.work_bytes = cap * 32;
}

// Grows the merge work area to hold `need` 32-byte units.
int ensure_work_cap(itokmc_handle* h, uint64_t need)
{
    if (need <= h->d.work_cap) return ITOKMC_OK;
    const uint64_t cap = std::max<uint64_t>(need + need / 4, h->d.work_cap * 2);
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    dfree(h, h->d.work);
    set_work(h, nullptr, 0);
    int rc = 0;
    unsigned char* p = reinterpret_cast<unsigned char*>(dalloc(h, cap * 32, &rc));
    if (rc) return rc;
    set_work(h, p, cap);
    return ITOKMC_OK;
}

// The field stream gets the highest priority: the solve is the longer of
// the two concurrent branches of a step, the particle kernels fill in.
cudaError_t create_field_stream(cudaStream_t* sf)
{
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return e;
    return cudaStreamCreateWithPriority(sf, cudaStreamNonBlocking, hi);
}

int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

// The step-size dependent constants: sqrt(2 D dt) and the FP32 form's
// drift and diffusion in cell units, for the electrons and (per species)
// for every particle block.
void set_step_consts(const itokmc_config* cfg, ik::Params& P, double dt)
{
    P.dt = dt;
    P.sdt = sqrt((2.0 * cfg->D) * dt);
    P.f_drift = (float)(-cfg->mu * dt / P.h[0]);
    P.f_diff = (float)(P.sdt / P.h[0]);
    const double sdt_ion = sqrt((2.0 * cfg->D_ion) * dt);
    const double cmu[3] = { -cfg->mu, cfg->mu_ion, -cfg->mu_ion };
    for (int s = 0; s < 3; ++s) {
        P.cmu_sp[s] = cmu[s];
        P.sdt_sp[s] = s == 0 ? P.sdt : sdt_ion;
        P.f_drift_sp[s] = s == 0 ? P.f_drift : (float)(cmu[s] * dt / P.h[0]);
        P.f_diff_sp[s] = (float)(P.sdt_sp[s] / P.h[0]);
    }
}

// Kernel parameters of a configuration (grid of n^3 cells per realization).
void fill_params(const itokmc_config* cfg, ik::Params& P)
{
    const int n = cfg->n[0];
    P.n = n; P.n3 = n * n * n; P.R = cfg->n_realizations; P.log2n = ilog2(n);
    P.S = cfg->mobile_ions ? 3 : 1;
    P.B = P.S * P.R;
    const uint32_t push_tags[3] = { ik::TAG_PUSH, ik::TAG_PUSH_POS, ik::TAG_PUSH_NEG };
    const uint32_t prod_tags[3] = { ik::TAG_PRODUCT, ik::TAG_PRODUCT_POS, ik::TAG_PRODUCT_NEG };
    for (int s = 0; s < 3; ++s) { P.push_tag_sp[s] = push_tags[s]; P.prod_tag_sp[s] = prod_tags[s]; }
    P.ppc = cfg->ppc; P.n_new = cfg->n_new; P.n_crit = cfg->n_crit; P.n_ssa = cfg->n_ssa; P.frac_bits = cfg->frac_bits;
    P.dep_win = ik::DEP_WIN_MAX;
    for (int a = 0; a < 3; ++a) {
        P.lo[a] = cfg->lo[a]; P.hi[a] = cfg->hi[a]; P.h[a] = (cfg->hi[a] - cfg->lo[a]) / n;
        P.rh[a] = 1.0 / P.h[a];
    }
    P.mu = cfg->mu; P.D = cfg->D; P.alpha_A = cfg->alpha_A; P.alpha_B = cfg->alpha_B; P.eta = cfg->eta;
    P.photon_ratio = cfg->photon_ratio; P.kappa_lo = cfg->kappa_lo; P.kappa_hi = cfg->kappa_hi; P.eps = cfg->eps;
    set_step_consts(cfg, P, cfg->dt);
    const double dV = (P.h[0] * P.h[1]) * P.h[2];
    P.k_ep = cfg->beta_ep / dV;
    P.k_np = cfg->beta_np / dV;
    P.E0 = cfg->E0;
    P.seed0 = cfg->seed0;
    P.step = 0;
    P.step_dev = nullptr;
}

int status_of_err(itokmc_handle* h, unsigned err)
{
    if (!err) return ITOKMC_OK;
    if (err & ik::DERR_CAPACITY) return fail(h, ITOKMC_ERR_CAPACITY, "particle, mover, photon or merge capacity exceeded");
    if (err & ik::DERR_OVERFLOW) return fail(h, ITOKMC_ERR_OVERFLOW, "weight or fixed-point overflow");
    if (err & ik::DERR_KMC) return fail(h, ITOKMC_ERR_KMC, "KMC iteration guard hit");
    if (err & ik::DERR_TIMEOUT) return fail(h, ITOKMC_ERR_TIMEOUT, "device wait timed out");
    return fail(h, ITOKMC_ERR_ARG, "invalid particle data (outside the domain, zero weight or bad realization)");
}

// Copies N (from cell_start[G]) and the counters to the pinned mirror and waits.
int readback(itokmc_handle* h)
{
    IK_CHECK(h, cudaMemcpyAsync(&h->rb->N, h->d.cell_start + h->Gp, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->s));
    IK_CHECK(h, cudaMemcpyAsync(&h->rb->ctr, h->d.ctr, sizeof(ik::Counters), cudaMemcpyDeviceToHost, h->s));
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    IK_CHECK(h, cudaGetLastError());
    h->N = h->rb->N;
    return ITOKMC_OK;
}

float elapsed(itokmc_handle* h, int a, int b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]) != cudaSuccess) { cudaGetLastError(); return -1.f; }
    return ms;
}

int transport_body(itokmc_handle* h)
{
    IK_CHECK(h, cudaEventRecord(h->ev[0], h->s));
    ik::launch_transport(h->P, h->d, h->N, h->s);
    ik::launch_transport_finish(h->P, h->d, h->N, h->Gp, h->s);
    ik::launch_rho(h->P, h->d, h->G, h->s);
    IK_CHECK(h, cudaEventRecord(h->ev[1], h->s));
    int rc = readback(h);
    if (rc) return rc;
    const ik::Counters& c = h->rb->ctr;
    h->st.n_movers = (int64_t)c.n_movers;
    // absorbed weight per particle block: electrons, then the ion species
    int64_t out[3] = { 0, 0, 0 };
    for (int b = 0; b < h->P.B; ++b) out[ik::species_of(h->P, b)] += (int64_t)c.outflow[b];
    h->st.outflow_weight = out[0];
    h->st.outflow_ion_pos = out[1];
    h->st.outflow_ion_neg = out[2];
    h->st.ms_transport = elapsed(h, 0, 1);
    return status_of_err(h, c.err);
}

int kmc_body(itokmc_handle* h)
{
    IK_CHECK(h, cudaEventRecord(h->ev[2], h->s));
    ik::launch_kmc(h->P, h->d, h->G, h->s);
    IK_CHECK(h, cudaEventRecord(h->ev[3], h->s));
    return cuda_check(h, cudaGetLastError(), "kmc launch");
}

int particles_body(itokmc_handle* h)
{
    IK_CHECK(h, cudaEventRecord(h->ev[4], h->s));
    // the photon list must hold every superphoton this step can emit
    IK_CHECK(h, cudaMemcpyAsync(&h->rb->ctr, h->d.ctr, sizeof(ik::Counters), cudaMemcpyDeviceToHost, h->s));
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    int rc = ensure_photo_cap(h, h->rb->ctr.photo_slots);
    if (rc) return rc;
    ik::launch_particles_a(h->P, h->d, h->G, h->s);
    // output count and merge work size are known after the merge scan
    uint64_t tail[2];
    uint32_t outn = 0;
    IK_CHECK(h, cudaMemcpyAsync(&tail[0], h->d.work_off + h->Gp, sizeof(uint64_t), cudaMemcpyDeviceToHost, h->s));
    IK_CHECK(h, cudaMemcpyAsync(&outn, h->d.out_start + h->Gp, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->s));
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    (void)tail[1];
    if (outn > h->cap) return fail(h, ITOKMC_ERR_CAPACITY, "particle capacity exceeded by the merge output");
    h->last_photo_slots = h->rb->ctr.photo_slots;
    h->last_work = tail[0];
    rc = ensure_work_cap(h, tail[0]);
    if (rc) return rc;
    ik::launch_particles_b(h->P, h->d, h->G, h->s);
    IK_CHECK(h, cudaEventRecord(h->ev[5], h->s));
    rc = readback(h);
    if (rc) return rc;
    const ik::Counters& c = h->rb->ctr;
    h->st.ionizations = (int64_t)c.ion;
    h->st.attachments = (int64_t)c.att;
    h->st.photon_emissions = (int64_t)c.phot;
    h->st.recombinations_ep = (int64_t)c.rec_ep;
    h->st.recombinations_np = (int64_t)c.rec_np;
    h->st.photons_absorbed_weight = (int64_t)c.absorbed_w;
    int64_t lost = 0;
    for (int r = 0; r < h->P.R; ++r) lost += (int64_t)c.lost[r];
    h->st.photons_lost_weight = lost;
    h->st.n_new_particles = (int64_t)c.n_photo;
    h->st.kmc_status = (c.err & ik::DERR_KMC) ? ITOKMC_ERR_KMC : 0;
    h->st.ms_kmc = elapsed(h, 2, 3);
    h->st.ms_particles = elapsed(h, 4, 5);
    h->st.merge_cells = (int64_t)c.merge_cells;
    h->st.merge_elements = (int64_t)c.merge_elems;
    h->st.merge_elements_sq = (int64_t)c.merge_elems2;
    h->st.merge_max_list = (int64_t)c.merge_maxm;
    return status_of_err(h, c.err);
}

// a5 on stream s into the field arrays E / E32 (the handle's own, or the
// next step's when the solve overlaps the particle stages).
int stage_field_on(itokmc_handle* h, cudaStream_t s, ik::E64* E, float4* E32, unsigned long long rho_absmax,
                   bool extrapolate = false)
{
    IK_CHECK(h, cudaEventRecord(h->ev[6], s));
    int cycles = 0;
    double rel = 0.0;
    const int st = ik::field_solve(h->P, h->d, h->d.phi_F > 0 ? 2 : h->field_prec, h->cfg.mg_rtol, h->cfg.mg_nu1,
                                   h->cfg.mg_nu2, rho_absmax, h->cfg.mg_max_cycles, s, &cycles, &rel, extrapolate);
    if (st == -3) return cuda_check(h, cudaGetLastError(), "field solve");
    ik::launch_efield_to(h->P, h->d, s, E, E32);
    IK_CHECK(h, cudaEventRecord(h->ev[7], s));
    IK_CHECK(h, cudaStreamSynchronize(s));
    IK_CHECK(h, cudaGetLastError());
    h->st.mg_cycles = cycles;
    h->st.mg_rel_residual = rel;
    h->st.ms_field = elapsed(h, 6, 7);
    if (st != 0) {
        char buf[160];
        snprintf(buf, sizeof buf, "multigrid stopped at %d cycles, relative residual %.3e", cycles, rel);
        return fail(h, ITOKMC_ERR_NOCONV, buf);
    }
    return ITOKMC_OK;
}

int stage_field(itokmc_handle* h) { return stage_field_on(h, h->s, h->d.E, h->d.E32, h->rb->ctr.rho_absmax); }

// The semi-implicit transport stage (Sec. 4.3, Sec. 4.7 steps 1-5): the
// conductivity of the start of the step, the diffusive substep, the charge of
// the diffused particles, the variable-coefficient solve for the field of
// the end of the step (into d.E), the advective substep, sort and deposit.
int semi_transport_body(itokmc_handle* h, int32_t* cycles_out, double* rel_out)
{
    if (h->P.S != 1) return fail(h, ITOKMC_ERR_ARG, "semi-implicit transport: ions as per-cell counts only");
    ik::Dev& d = h->d;
    if (d.mixed || d.phi_F > 0)
        return fail(h, ITOKMC_ERR_ARG, "semi-implicit transport: FP64 form only");
    // no work of an overlapped field solve may still be in flight
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    if (h->sf) IK_CHECK(h, cudaStreamSynchronize(h->sf));
    int rc = 0;
    for (int l = 0; l < d.nlev && !rc; ++l)
        if (!d.vc[l].c) {
            const size_t cells = (size_t)h->P.R * d.lev[l].n * d.lev[l].n * d.lev[l].n;
            ik::VCLevel& V = d.vc[l];
            V.c = dalloc_n<double>(h, cells, &rc);
            V.fx = dalloc_n<double>(h, cells, &rc);
            V.fy = dalloc_n<double>(h, cells, &rc);
            V.fz = dalloc_n<double>(h, cells, &rc);
            V.dg = dalloc_n<double>(h, cells, &rc);
            V.idg = dalloc_n<double>(h, cells, &rc);
        }
    if (rc) return rc;
    IK_CHECK(h, cudaEventRecord(h->ev[0], h->s));
    ik::launch_deposit_only(h->P, d, h->N, h->s);       // n_e of the start of the step
    ik::launch_semi_coef(h->P, d, d.vc[0].c, h->s);
    ik::launch_diffuse(h->P, d, h->N, h->s);            // X+ into recB
    ik::launch_deposit_B(h->P, d, h->N, h->s);
    IK_CHECK(h, cudaMemsetAsync(d.ctr, 0, sizeof(ik::Counters), h->s));
    ik::launch_rho(h->P, d, h->G, h->s);                // rho+
    rc = readback(h);
    if (rc) return rc;
    rc = status_of_err(h, h->rb->ctr.err);
    if (rc) return rc;
    int cycles = 0;
    double rel = 0.0;
    const int st = ik::field_solve_vc(h->P, d, d.norm_out, d.norm_host, h->cfg.mg_rtol, h->cfg.mg_nu1, h->cfg.mg_nu2,
                                      h->cfg.mg_max_cycles, h->s, &cycles, &rel);
    if (cycles_out) *cycles_out = cycles;
    if (rel_out) *rel_out = rel;
    h->st.mg_cycles = cycles;
    h->st.mg_rel_residual = rel;
    if (st == -3) return cuda_check(h, cudaGetLastError(), "semi-implicit field solve");
    if (st != 0) return fail(h, ITOKMC_ERR_NOCONV, "semi-implicit field: multigrid did not reach mg_rtol");
    ik::launch_advect(h->P, d, h->N, h->s);
    ik::launch_transport_finish(h->P, d, h->N, h->Gp, h->s);
    ik::launch_rho(h->P, d, h->G, h->s);
    IK_CHECK(h, cudaEventRecord(h->ev[1], h->s));
    rc = readback(h);
    if (rc) return rc;
    const ik::Counters& c = h->rb->ctr;
    h->st.n_movers = (int64_t)c.n_movers;
    // absorbed weight per particle block: electrons, then the ion species
    int64_t out[3] = { 0, 0, 0 };
    for (int b = 0; b < h->P.B; ++b) out[ik::species_of(h->P, b)] += (int64_t)c.outflow[b];
    h->st.outflow_weight = out[0];
    h->st.outflow_ion_pos = out[1];
    h->st.outflow_ion_neg = out[2];
    h->st.ms_transport = elapsed(h, 0, 1);
    return status_of_err(h, c.err);
}

// One full step.  After the transport stage has formed rho, the field of the
// next step is solved on the field stream by a host thread while this
// thread runs KMC and the particle stages (they read the current field; the
// solve writes the next one); the two fields swap at the end.
// Stage order.  The KMC reads X_e of the last deposit, the particles stage
// the firings of the last KMC and the cell offsets of the last transport, so
// each stage runs only on the state the stages before it produced from the
// current particles: a transport (either coupling) may run at any time; the
// KMC after a transport, and again on the same transported state; the
// particles stage once after a KMC, after which the particles have changed
// and the next KMC needs a new transport.  h->stage is 0 (no deposit of the
// current particles), 1 (transported) or 2 (KMC done); replacing the
// particles (set, seed, load) returns it to 0.
int stage_transport(itokmc_handle* h)
{
    h->stage = 0;
    const int rc = transport_body(h);
    if (!rc) h->stage = 1;
    return rc;
}

int stage_semi_transport(itokmc_handle* h, int32_t* cycles_out, double* rel_out)
{
    h->stage = 0;
    const int rc = semi_transport_body(h, cycles_out, rel_out);
    if (!rc) h->stage = 1;
    return rc;
}

int stage_kmc(itokmc_handle* h)
{
    if (h->stage < 1) return fail(h, ITOKMC_ERR_ARG, "stage order: the KMC needs a transport stage first");
    const int rc = kmc_body(h);
    h->stage = rc ? 0 : 2;
    return rc;
}

int stage_particles(itokmc_handle* h)
{
    if (h->stage != 2) return fail(h, ITOKMC_ERR_ARG, "stage order: the particles stage needs a KMC after a transport");
    h->stage = 0;
    return particles_body(h);
}


// ---------------------------------------------------------------- graph steps
// A whole explicit step (transport, deposit and charge, the field solve on
// its own stream beside KMC, products, photons and merge) captured once as a
// CUDA graph and replayed: one launch per step, no host synchronisation
// inside it.  The particle count is read on the device (grids cover the
// capacity), the step counter from device memory, the field solve runs a
// fixed number of cycles (the count the last host-driven solve needed) and
// leaves its residual norms for a check after the step.  The device buffers
// a step swaps (offsets, records, field) cycle with a short period, so a
// graph is cached per starting state, with the state it leaves.
struct DevState {
    uint32_t *cell_start, *cell_start_B, *out_start, *cellA32, *cellB32, *photo_sorted;
    ik::P64 *recA, *recB;
    ik::P32 *rA32, *rB32;
    ik::E64 *E, *E_next;
    float4 *E32, *E32_next;
    ik::Photo* photos;
    unsigned char* work;
    uint64_t work_cap, work_bytes;
    uint32_t photo_cap;
    int phi_F;
    bool have_prev;
};

DevState snapshot(const ik::Dev& d)
{
    DevState x;
    std::memset(&x, 0, sizeof x);
    x.cell_start = d.cell_start; x.cell_start_B = d.cell_start_B; x.out_start = d.out_start;
    x.cellA32 = d.cellA32; x.cellB32 = d.cellB32; x.photo_sorted = d.photo_sorted;
    x.recA = d.recA; x.recB = d.recB; x.rA32 = d.rA32; x.rB32 = d.rB32;
    x.E = d.E; x.E_next = d.E_next; x.E32 = d.E32; x.E32_next = d.E32_next;
    x.photos = d.photos; x.work = d.work; x.work_cap = d.work_cap; x.work_bytes = d.work_bytes;
    x.photo_cap = d.photo_cap; x.phi_F = d.phi_F; x.have_prev = d.have_prev;
    return x;
}

void apply(ik::Dev& d, const DevState& x)
{
    d.cell_start = x.cell_start; d.cell_start_B = x.cell_start_B; d.out_start = x.out_start;
    d.cellA32 = x.cellA32; d.cellB32 = x.cellB32; d.photo_sorted = x.photo_sorted;
    d.recA = x.recA; d.recB = x.recB; d.rA32 = x.rA32; d.rB32 = x.rB32;
    d.E = x.E; d.E_next = x.E_next; d.E32 = x.E32; d.E32_next = x.E32_next;
    d.photos = x.photos; d.work = x.work; d.work_cap = x.work_cap; d.work_bytes = x.work_bytes;
    d.photo_cap = x.photo_cap; d.phi_F = x.phi_F; d.have_prev = x.have_prev;
}

bool same(const DevState& a, const DevState& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

}  // namespace

struct itokmc_handle::GraphEntry {
    DevState before, after;
    int cycles;
    uint32_t nbound;
    cudaGraphExec_t exec;
};

namespace {

void drop_graphs(itokmc_handle* h)
{
    for (auto* e : h->graphs) {
        if (e->exec) cudaGraphExecDestroy(e->exec);
        delete e;
    }
    h->graphs.clear();
}

// The launches of one step, issued on the capture stream (no waits).
void graph_launches(itokmc_handle* h, int prec)
{
    ik::Dev& d = h->d;
    ik::Params& P = h->P;
    cudaStream_t s = h->scap;
    const uint32_t* Ndev = d.cell_start + h->Gp;          // the count before the step
    cudaMemcpyAsync(d.step_dev, &h->rb->step, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    ik::launch_transport(P, d, h->graph_nbound, s, Ndev);
    ik::launch_transport_finish(P, d, h->graph_nbound, h->Gp, s, Ndev);
    ik::launch_rho(P, d, h->G, s);
    cudaEventRecord(h->fork, s);
    cudaStreamWaitEvent(h->sf, h->fork, 0);
    ik::field_solve_fixed(P, d, prec, h->cfg.mg_nu1, h->cfg.mg_nu2, h->graph_cycles, h->sf);
    ik::launch_efield_to(P, d, h->sf, d.E_next, d.E32_next);
    ik::launch_kmc(P, d, h->G, s);
    ik::launch_particles_a(P, d, h->G, s);
    ik::launch_particles_b(P, d, h->G, s);
    cudaEventRecord(h->join, h->sf);
    cudaStreamWaitEvent(s, h->join, 0);
    cudaMemcpyAsync(&h->rb->ctr, d.ctr, sizeof(ik::Counters), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&h->rb->N, d.cell_start + h->Gp, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&h->rb->work_need, d.work_off + h->Gp, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(d.norm_host, d.norm_out, 2 * (size_t)P.R * sizeof(double), cudaMemcpyDeviceToHost, s);
    std::swap(d.E, d.E_next);
    std::swap(d.E32, d.E32_next);
}

// Whether the next step may be a replayed one: explicit coupling at a fixed
// step size, at a step boundary, after a host-driven step has measured the
// field's cycle count and the buffers' use, with headroom in every buffer a
// step can fill (particles at most 2/3 of the capacity, photon slots and
// merge work at most half their buffers, and a fixed-point potential scale
// that holds for four times the last charge).
bool graph_eligible(itokmc_handle* h)
{
    const itokmc_config& c = h->cfg;
    if (!c.graph_step || c.dt_adapt || c.coupling != ITOKMC_EXPLICIT || h->stage != 0) return false;
    if (h->steps_done < 1 || h->graph_cycles < 1 || h->graph_cycles > c.mg_max_cycles) return false;
    if ((uint64_t)h->N * 3 > (uint64_t)h->cap * 2 || h->N == 0) return false;
    // the transport grids cover the next power of two of the count (at most
    // twice the work of exact grids; a count beyond it is a new graph)
    uint64_t nb = 256;
    while (nb < h->N) nb <<= 1;
    h->graph_nbound = (uint32_t)std::min<uint64_t>(nb, h->cap);
    // photon and merge-work buffers grow here, between steps, to twice the
    // last use (a new buffer is a new starting state: its own graph)
    if (ensure_photo_cap(h, 2 * h->last_photo_slots + 1024) || ensure_work_cap(h, 2 * h->last_work + 1024)) return false;
    // the fixed-point potential's scale: lowered here, if need be, to one that
    // holds for four times the last charge (the host-driven solve lowers it
    // the same way when the charge requires)
    if (h->d.phi_F > 0)
        ik::lower_phi_scale(h->P, h->d, ik::phi_fixed_bits(ik::phi_bound(h->P, 4 * h->last_rho_absmax + 1)), h->s);
    return h->d.have_prev;
}

int graph_step(itokmc_handle* h)
{
    ik::Dev& d = h->d;
    const int prec = d.phi_F > 0 ? 2 : h->field_prec;
    const DevState cur = snapshot(d);
    itokmc_handle::GraphEntry* e = nullptr;
    for (auto* x : h->graphs)
        if (x->cycles == h->graph_cycles && x->nbound == h->graph_nbound && same(x->before, cur)) { e = x; break; }
    h->rb->step = (uint32_t)h->step;
    if (!e) {
        if (h->graphs.size() >= 12) drop_graphs(h);
        IK_CHECK(h, cudaStreamSynchronize(h->s));
        const bool dc = d.direct_cycles;
        d.direct_cycles = true;                  // V-cycles as plain launches inside the capture
        h->P.step_dev = d.step_dev;
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(h->scap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            graph_launches(h, prec);
            ce = cudaStreamEndCapture(h->scap, &g);
        }
        h->P.step_dev = nullptr;
        d.direct_cycles = dc;
        const DevState after = snapshot(d);
        apply(d, cur);
        cudaGraphExec_t ex = nullptr;
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (ce != cudaSuccess) return cuda_check(h, ce, "step graph capture");
        e = new itokmc_handle::GraphEntry{ cur, after, h->graph_cycles, h->graph_nbound, ex };
        h->graphs.push_back(e);
    }
    IK_CHECK(h, cudaGraphLaunch(e->exec, h->s));
    ++h->st.graph_steps;
    apply(d, e->after);
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    IK_CHECK(h, cudaGetLastError());
    // the step's results and checks
    const ik::Counters& c = h->rb->ctr;
    h->N = h->rb->N;
    h->stage = 0;
    h->last_photo_slots = c.photo_slots;
    h->last_work = h->rb->work_need;
    h->last_rho_absmax = c.rho_absmax;
    h->st.n_movers = (int64_t)c.n_movers;
    int64_t out[3] = { 0, 0, 0 };
    for (int b = 0; b < h->P.B; ++b) out[ik::species_of(h->P, b)] += (int64_t)c.outflow[b];
    h->st.outflow_weight = out[0];
    h->st.outflow_ion_pos = out[1];
    h->st.outflow_ion_neg = out[2];
    h->st.ionizations = (int64_t)c.ion;
    h->st.attachments = (int64_t)c.att;
    h->st.photon_emissions = (int64_t)c.phot;
    h->st.recombinations_ep = (int64_t)c.rec_ep;
    h->st.recombinations_np = (int64_t)c.rec_np;
    h->st.photons_absorbed_weight = (int64_t)c.absorbed_w;
    int64_t lost = 0;
    for (int r = 0; r < h->P.R; ++r) lost += (int64_t)c.lost[r];
    h->st.photons_lost_weight = lost;
    h->st.n_new_particles = (int64_t)c.n_photo;
    h->st.kmc_status = (c.err & ik::DERR_KMC) ? ITOKMC_ERR_KMC : 0;
    h->st.merge_cells = (int64_t)c.merge_cells;
    h->st.merge_elements = (int64_t)c.merge_elems;
    h->st.merge_elements_sq = (int64_t)c.merge_elems2;
    h->st.merge_max_list = (int64_t)c.merge_maxm;
    h->st.ms_transport = h->st.ms_kmc = h->st.ms_particles = h->st.ms_field = 0.0;
    if (c.err) return status_of_err(h, c.err);
    if (h->N > h->cap) return fail(h, ITOKMC_ERR_CAPACITY, "particle capacity exceeded by the merge output");
    int rc = ensure_work_cap(h, h->last_work);
    if (!rc) rc = ensure_photo_cap(h, h->last_photo_slots);
    if (rc) return rc;
    // the field: tolerance reached and the fixed-point scale still valid, else
    // the host-driven solve continues from the replayed one
    double worst = 0.0;
    bool done = true;
    for (int r = 0; r < h->P.R; ++r) {
        const double rn = std::sqrt(d.norm_host[2 * r]), bn = std::sqrt(d.norm_host[2 * r + 1]);
        const double rel = bn > 0.0 ? rn / bn : rn;
        if (rel > worst || !(rel == rel)) worst = rel;
        if (!(rn <= h->cfg.mg_rtol * bn)) done = false;
    }
    const bool scale_ok = d.phi_F == 0 || ik::phi_fixed_bits(ik::phi_bound(h->P, c.rho_absmax)) >= d.phi_F;
    h->st.mg_cycles = h->graph_cycles;
    h->st.mg_rel_residual = worst;
    if (!done || !scale_ok) {
        rc = stage_field_on(h, h->s, d.E, d.E32, c.rho_absmax, false);
        if (rc) return rc;
        h->graph_cycles = std::max(h->graph_cycles, h->st.mg_cycles + h->graph_cycles);
    }
    return ITOKMC_OK;
}

int full_step(itokmc_handle* h)
{
    int rc = stage_transport(h);
    if (rc) return rc;
    IK_CHECK(h, cudaEventRecord(h->fork, h->s));
    IK_CHECK(h, cudaStreamWaitEvent(h->sf, h->fork, 0));
    const unsigned long long amax = h->rb->ctr.rho_absmax;
    int frc = ITOKMC_OK;
    std::string ferr;
    std::thread field([h, amax, &frc, &ferr]() {
        if (cudaSetDevice(h->device) != cudaSuccess) {
            frc = ITOKMC_ERR_CUDA;
            ferr = "field thread: cudaSetDevice";
            return;
        }
        frc = stage_field_on(h, h->sf, h->d.E_next, h->d.E32_next, amax, true);
        if (frc) {
            std::lock_guard<std::mutex> lk(h->emtx);
            ferr = h->err;
        }
    });
    rc = stage_kmc(h);
    if (!rc) rc = stage_particles(h);
    field.join();
    IK_CHECK(h, cudaEventRecord(h->join, h->sf));
    IK_CHECK(h, cudaStreamWaitEvent(h->s, h->join, 0));
    if (rc) return rc;
    if (frc) return fail(h, frc, ferr);
    std::swap(h->d.E, h->d.E_next);
    std::swap(h->d.E32, h->d.E32_next);
    h->graph_cycles = h->st.mg_cycles;
    h->last_rho_absmax = amax;
    return ITOKMC_OK;
}

// The adaptive step size (dt_adapt): dt 2^-j, j the smallest >= 0 with the
// step under every active bound, from the largest |E| of the field that
// pushes the particles and the densest cell of the last deposit; never
// below the largest such step not under dt_min.  Sets the step-dependent
// kernel constants.
int choose_step(itokmc_handle* h)
{
    ik::Params& P = h->P;
    const itokmc_config& c = h->cfg;
    double dt = c.dt;
    if (c.dt_adapt) {
        unsigned long long* m = reinterpret_cast<unsigned long long*>(h->d.norm_out);   // 2 words of scratch
        ik::launch_step_maxima(P, h->d, m, h->s);
        unsigned long long hm[2] = { 0, 0 };
        IK_CHECK(h, cudaMemcpyAsync(hm, m, sizeof hm, cudaMemcpyDeviceToHost, h->s));
        IK_CHECK(h, cudaStreamSynchronize(h->s));
        double Emax;
        std::memcpy(&Emax, &hm[0], sizeof Emax);
        const double hcell = P.h[0];
        double b = INFINITY;
        if (c.cfl > 0.0 && c.mu * Emax > 0.0) b = std::min(b, c.cfl * hcell / (c.mu * Emax));
        if (c.cfl > 0.0 && c.D > 0.0) b = std::min(b, (c.cfl * hcell) * (c.cfl * hcell) / (2.0 * c.D));
        if (c.coupling == ITOKMC_EXPLICIT && c.drt_factor > 0.0 && hm[1] > 0) {
            const double dV = (hcell * hcell) * hcell;
            const double nmax = (double)hm[1] * std::ldexp(1.0, -3 * P.frac_bits) / dV;
            b = std::min(b, c.drt_factor * 8.8541878128e-12 / (1.602176634e-19 * c.mu * nmax));
        }
        if (c.ion_factor > 0.0 && Emax > 0.0) {
            const double k = c.alpha_A * std::exp(-c.alpha_B / Emax) * (c.mu * Emax);
            if (k > 0.0) b = std::min(b, c.ion_factor / k);
        }
        int j = 0;
        while (j < 62 && std::ldexp(c.dt, -j) > b && std::ldexp(c.dt, -(j + 1)) >= c.dt_min) ++j;
        dt = std::ldexp(c.dt, -j);
    }
    set_step_consts(&c, P, dt);
    h->st.dt_last = dt;
    return ITOKMC_OK;
}

// One semi-implicit step (Sec. 4.7): the semi-implicit transport stage
// solves the field of the end of the step, with which KMC and the particle
// stages then run; nothing overlaps (the next step's field is solved inside
// the next transport stage).
int semi_step(itokmc_handle* h)
{
    int rc = stage_semi_transport(h, nullptr, nullptr);
    if (!rc) rc = stage_kmc(h);
    if (!rc) rc = stage_particles(h);
    return rc;
}

}  // namespace

namespace ik {
int handle_view(itokmc_handle* h, HandleView* v)
{
    IK_GUARD(h);
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    if (h->sf) IK_CHECK(h, cudaStreamSynchronize(h->sf));
    *v = HandleView{ &h->cfg, &h->P, &h->d, h->s, &h->N, h->cap, &h->step, h->G, h->field_prec, h->Gp, &h->stage };
    return ITOKMC_OK;
}
int handle_fail(itokmc_handle* h, int code, const char* msg) { return fail(h, code, msg); }
int handle_solve_field(itokmc_handle* h) { return itokmc_solve_field(h); }
}  // namespace ik

extern "C" {

int itokmc_config_defaults(itokmc_config* c)
{
    if (!c) return ITOKMC_ERR_ARG;
    memset(c, 0, sizeof(*c));
    c->n_realizations = 1;
    c->eps = INFINITY;
    c->ppc = 8;
    c->n_new = 64;
    c->n_crit = 5;
    c->n_ssa = 10;
    c->frac_bits = 10;
    c->precision = ITOKMC_FP64;
    c->field_precision = -1;
    c->mg_rtol = 1e-10;
    c->mg_nu1 = 2;
    c->mg_nu2 = 2;
    c->mg_max_cycles = 64;
    c->kappa_lo = 520.0;
    c->kappa_hi = 3.0e4;
    return ITOKMC_OK;
}

int itokmc_init(const itokmc_config* cfg, itokmc_handle** out)
{
    if (!cfg || !out) return fail(nullptr, ITOKMC_ERR_ARG, "NULL argument");
    *out = nullptr;
    const int n = cfg->n[0];
    if (n < 8 || (n & (n - 1)) || cfg->n[1] != n || cfg->n[2] != n || n > 1024)
        return fail(nullptr, ITOKMC_ERR_ARG, "grid must be n^3 with n a power of two in [8, 1024]");
    const int R = cfg->n_realizations;
    if (R < 1 || R > ik::MAX_R) return fail(nullptr, ITOKMC_ERR_ARG, "n_realizations out of range");
    const uint64_t G = (uint64_t)R * n * n * n;
    if (G > ik::KEY_MASK) return fail(nullptr, ITOKMC_ERR_ARG, "too many cells (R n^3 must be < 2^30)");
    const double h0 = (cfg->hi[0] - cfg->lo[0]) / n;
    for (int a = 0; a < 3; ++a) {
        if (!(cfg->hi[a] > cfg->lo[a])) return fail(nullptr, ITOKMC_ERR_ARG, "hi must exceed lo");
        if ((cfg->hi[a] - cfg->lo[a]) / n != h0) return fail(nullptr, ITOKMC_ERR_ARG, "cells must be cubes");
    }
    if (!(cfg->dt > 0) || cfg->D < 0 || cfg->mu < 0) return fail(nullptr, ITOKMC_ERR_ARG, "dt, mu, D");
    if (cfg->ppc < 1 || cfg->ppc > 256 || (cfg->ppc & (cfg->ppc - 1)))
        return fail(nullptr, ITOKMC_ERR_ARG, "ppc must be a power of two <= 256");
    if (cfg->n_new < 1 || cfg->n_new > 64) return fail(nullptr, ITOKMC_ERR_ARG, "n_new in [1, 64]");
    if (cfg->frac_bits < 1 || cfg->frac_bits > 10) return fail(nullptr, ITOKMC_ERR_ARG, "frac_bits in [1, 10]");
    if (cfg->n_ssa < 1 || cfg->n_crit < 0) return fail(nullptr, ITOKMC_ERR_ARG, "n_ssa, n_crit");
    if (cfg->precision != ITOKMC_FP64 && cfg->precision != ITOKMC_MIXED)
        return fail(nullptr, ITOKMC_ERR_ARG, "precision");
    if (cfg->field_precision != -1 && cfg->field_precision != ITOKMC_FP64 && cfg->field_precision != ITOKMC_MIXED)
        return fail(nullptr, ITOKMC_ERR_ARG, "field_precision: -1, ITOKMC_FP64 or ITOKMC_MIXED");
    if (cfg->particle_capacity < 1 || cfg->particle_capacity > 0x7fff0000ll)
        return fail(nullptr, ITOKMC_ERR_ARG, "particle_capacity in [1, 2^31)");
    if (cfg->photon_ratio > 0 && !(cfg->kappa_hi >= cfg->kappa_lo && cfg->kappa_lo > 0))
        return fail(nullptr, ITOKMC_ERR_ARG, "kappa range");
    if (!(cfg->alloc == nullptr) != !(cfg->free_fn == nullptr))
        return fail(nullptr, ITOKMC_ERR_ARG, "alloc and free_fn must be given together");
    if (cfg->n_blobs < 0 || (cfg->n_blobs > 0 && !cfg->blobs))
        return fail(nullptr, ITOKMC_ERR_ARG, "n_blobs >= 0 with a blob array");
    if (cfg->dt_adapt != 0 && cfg->dt_adapt != 1) return fail(nullptr, ITOKMC_ERR_ARG, "dt_adapt: 0 or 1");
    if (cfg->dt_adapt && !(cfg->dt_min > 0.0 && cfg->dt_min <= cfg->dt && cfg->cfl >= 0.0 && cfg->drt_factor >= 0.0 &&
                           cfg->ion_factor >= 0.0))
        return fail(nullptr, ITOKMC_ERR_ARG, "adaptive step: 0 < dt_min <= dt, cfl, drt_factor, ion_factor >= 0");
    if (!(cfg->beta_ep >= 0.0 && cfg->beta_np >= 0.0 && std::isfinite(cfg->beta_ep) && std::isfinite(cfg->beta_np)))
        return fail(nullptr, ITOKMC_ERR_ARG, "recombination coefficients: finite, >= 0");
    if (cfg->mobile_ions != 0 && cfg->mobile_ions != 1) return fail(nullptr, ITOKMC_ERR_ARG, "mobile_ions: 0 or 1");
    if (cfg->mobile_ions && !(cfg->mu_ion >= 0.0 && cfg->D_ion >= 0.0 && std::isfinite(cfg->mu_ion) &&
                              std::isfinite(cfg->D_ion)))
        return fail(nullptr, ITOKMC_ERR_ARG, "mobile ions: finite mu_ion, D_ion >= 0");
    if (cfg->mobile_ions && cfg->coupling != ITOKMC_EXPLICIT)
        return fail(nullptr, ITOKMC_ERR_ARG, "mobile ions: explicit coupling only");
    if (cfg->mobile_ions && 3 * R > ik::MAX_R) return fail(nullptr, ITOKMC_ERR_ARG, "mobile ions: 3 R particle blocks > MAX_R");
    if (cfg->coupling != ITOKMC_EXPLICIT && cfg->coupling != ITOKMC_SEMI_IMPLICIT)
        return fail(nullptr, ITOKMC_ERR_ARG, "coupling: ITOKMC_EXPLICIT or ITOKMC_SEMI_IMPLICIT");
    if (cfg->coupling == ITOKMC_SEMI_IMPLICIT &&
        (cfg->precision != ITOKMC_FP64 || (cfg->field_precision != -1 && cfg->field_precision != ITOKMC_FP64)))
        return fail(nullptr, ITOKMC_ERR_ARG, "semi-implicit coupling: FP64 form only");

    itokmc_handle* h = new itokmc_handle();
    h->cfg = *cfg;
    h->s = (cudaStream_t)cfg->stream;
    h->G = G;
    h->cap = (uint32_t)cfg->particle_capacity;
    h->field_prec = cfg->field_precision < 0 ? cfg->precision : cfg->field_precision;
    ik::Params& P = h->P;
    fill_params(cfg, P);
    h->Gp = G * (uint64_t)P.S;
    const uint64_t Gp = h->Gp;
    h->st.dt_last = cfg->dt;

    int rc = 0;
    ik::Dev& d = h->d;
    const size_t cap = h->cap;
    d.mover_cap = h->cap;
    d.photo_cap = (uint32_t)std::max<size_t>(1u << 16, cap / 4);
    d.work_cap = std::max<uint64_t>(3ull << 20, 2 * (uint64_t)cap + 16);
    d.mixed = cfg->precision == ITOKMC_MIXED;
    // mixed field form: fixed-point potential and right-hand side
    d.phi_F = h->field_prec == ITOKMC_MIXED ? ik::phi_fixed_bits(ik::phi_bound(P, 0)) : 0;
    if (d.mixed) {
        d.rA32 = dalloc_n<ik::P32>(h, cap, &rc);
        d.rB32 = dalloc_n<ik::P32>(h, cap, &rc);
        d.cellA32 = dalloc_n<uint32_t>(h, cap, &rc);
        d.cellB32 = dalloc_n<uint32_t>(h, cap, &rc);
    } else {
        d.recA = dalloc_n<ik::P64>(h, cap, &rc);
        d.recB = dalloc_n<ik::P64>(h, cap, &rc);
    }
    d.keyB = dalloc_n<uint32_t>(h, cap, &rc);
    // particle-cell arrays: one block of n^3 per species and realization
    d.cell_start = dalloc_n<uint32_t>(h, Gp + 1, &rc);
    d.cell_start_B = dalloc_n<uint32_t>(h, Gp + 1, &rc);
    d.out_start = dalloc_n<uint32_t>(h, Gp + 1, &rc);
    d.cnt_new = dalloc_n<int32_t>(h, Gp, &rc);
    d.in_cnt = dalloc_n<int32_t>(h, Gp, &rc);
    d.in_before = dalloc_n<int32_t>(h, Gp, &rc);
    d.cursor = dalloc_n<int32_t>(h, Gp, &rc);
    d.delta = dalloc_n<int64_t>(h, Gp, &rc);
    d.in_off = dalloc_n<uint32_t>(h, Gp + 1, &rc);
    const size_t nblk = (cap + ik::TPB - 1) / ik::TPB + 1;
    d.blk_stay = dalloc_n<uint32_t>(h, nblk, &rc);
    d.blk_prefix = dalloc_n<uint32_t>(h, nblk, &rc);
    d.movers = dalloc_n<ik::Mover>(h, cap, &rc);
    d.mover_sorted = dalloc_n<uint32_t>(h, cap, &rc);
    d.ne_fix = dalloc_n<unsigned long long>(h, Gp, &rc);
    d.Xe = dalloc_n<unsigned long long>(h, Gp, &rc);
    d.gain = dalloc_n<int64_t>(h, Gp, &rc);
    d.step_dev = dalloc_n<uint32_t>(h, 1, &rc);
    d.Npos = dalloc_n<int64_t>(h, G, &rc);
    d.Nneg = dalloc_n<int64_t>(h, G, &rc);
    d.rho = dalloc_n<int64_t>(h, G, &rc);
    // FP64 form: FP64 field (push, KMC); mixed form: FP32 field only
    if (d.mixed) {
        d.E32 = dalloc_n<float4>(h, G, &rc);
        d.E32_next = dalloc_n<float4>(h, G, &rc);
    } else {
        d.E = dalloc_n<ik::E64>(h, G, &rc);
        d.E_next = dalloc_n<ik::E64>(h, G, &rc);
    }
    d.fired = dalloc_n<int64_t>(h, 5 * G, &rc);
    d.stage = dalloc_n<double>(h, 3 * G, &rc);
    d.phi_prev = dalloc_n<double>(h, G, &rc);
    d.photos = dalloc_n<ik::Photo>(h, d.photo_cap, &rc);
    d.photo_sorted = dalloc_n<uint32_t>(h, d.photo_cap, &rc);
    d.photo_cnt = dalloc_n<int32_t>(h, G, &rc);
    d.photo_cursor = dalloc_n<int32_t>(h, G, &rc);
    d.photo_w = dalloc_n<unsigned long long>(h, G, &rc);
    d.photo_off = dalloc_n<uint32_t>(h, Gp + 1, &rc);
    d.work_off = dalloc_n<uint64_t>(h, Gp + 1, &rc);
    d.small_list = dalloc_n<uint32_t>(h, Gp, &rc);
    d.mid_list = dalloc_n<uint32_t>(h, Gp, &rc);
    d.big_list = dalloc_n<uint32_t>(h, Gp, &rc);
    d.list_n = dalloc_n<uint32_t>(h, 4, &rc);
    d.pc_list = dalloc_n<uint32_t>(h, G, &rc);
    set_work(h, reinterpret_cast<unsigned char*>(dalloc(h, d.work_cap * 32, &rc)), d.work_cap);
    const size_t se = 2 * std::max(std::max(ik::scan_scratch_elems(Gp, 6), ik::scan_scratch_elems(nblk, 3)),
                                   ik::radix_scratch_elems(h->cap));
    d.scan_blk = dalloc_n<long long>(h, se, &rc);
    d.scan_blk_elems = se;
    d.ctr = dalloc_n<ik::Counters>(h, 1, &rc);
    d.sort_tmp = dalloc_n<uint32_t>(h, 4 * cap, &rc);
    // multigrid hierarchy down to 4^3
    int l = 0;
    for (int m = n; m >= 4 && l < ik::MAX_LEVELS; m >>= 1, ++l) {
        ik::MGLevel& L = d.lev[l];
        const size_t cells = (size_t)R * m * m * m;
        L.n = m;
        L.h = P.h[0] * (double)(n / m);
        L.phi = dalloc_n<double>(h, cells, &rc);
        L.rhs = dalloc_n<double>(h, cells, &rc);
        L.res = nullptr;
        L.phi32 = dalloc_n<float>(h, cells, &rc);
        L.rhs32 = dalloc_n<float>(h, cells, &rc);
    }
    d.nlev = l;
    const size_t nb = (size_t)R * n * n * n / 256 + 16;
    d.norm_part = dalloc_n<double>(h, 2 * nb, &rc);
    d.norm_out = dalloc_n<double>(h, 2 * R, &rc);
    if (!rc && cudaMallocHost(reinterpret_cast<void**>(&h->rb), sizeof(*h->rb)) != cudaSuccess)
        rc = fail(h, ITOKMC_ERR_OOM, "pinned host buffer");
    if (!rc && cudaMallocHost(reinterpret_cast<void**>(&d.norm_host), 2 * R * sizeof(double)) != cudaSuccess)
        rc = fail(h, ITOKMC_ERR_OOM, "pinned host buffer");
    for (int e = 0; e < 8 && !rc; ++e)
        if (cudaEventCreate(&h->ev[e]) != cudaSuccess) rc = fail(h, ITOKMC_ERR_CUDA, "event create");
    if (!rc && (cudaGetDevice(&h->device) != cudaSuccess ||
                create_field_stream(&h->sf) != cudaSuccess ||
                cudaStreamCreateWithFlags(&d.side, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&d.side_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&d.side_join, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess ||
                cudaStreamCreateWithFlags(&h->scap, cudaStreamNonBlocking) != cudaSuccess))
        rc = fail(h, ITOKMC_ERR_CUDA, "field stream");
    if (!rc) ik::launch_zig_init(h->s);
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->s), "init sync");
    if (rc) {
        ik::set_global_error(h->err.c_str());
        itokmc_destroy(h);
        return rc;
    }
    // initial seeds from the configuration: sample, deposit, initial field
    if (cfg->n_blobs > 0) {
        rc = itokmc_seed_blobs(h, cfg->blobs, cfg->n_blobs, cfg->seed_flags);
        if (!rc) rc = itokmc_solve_field(h);
        if (rc) {
            ik::set_global_error(h->err.c_str());
            itokmc_destroy(h);
            return rc;
        }
    }
    h->cfg.blobs = nullptr;           // read during init only
    h->cfg.n_blobs = 0;
    *out = h;
    return ITOKMC_OK;
}

int itokmc_destroy(itokmc_handle* h)
{
    if (!h) return ITOKMC_OK;
    cudaStreamSynchronize(h->s);
    cudaGetLastError();
    for (void* p : h->allocs) {
        if (h->cfg.free_fn) h->cfg.free_fn(p, h->cfg.alloc_ctx);
        else cudaFreeAsync(p, h->s);
    }
    cudaStreamSynchronize(h->s);
    if (h->sf) {
        cudaStreamSynchronize(h->sf);
        cudaStreamDestroy(h->sf);
    }
    for (auto& gx : h->d.vgraph)
        if (gx) cudaGraphExecDestroy(gx);
    drop_graphs(h);
    if (h->scap) cudaStreamDestroy(h->scap);
    if (h->d.side) {
        cudaStreamSynchronize(h->d.side);
        cudaStreamDestroy(h->d.side);
    }
    if (h->d.side_fork) cudaEventDestroy(h->d.side_fork);
    if (h->d.side_join) cudaEventDestroy(h->d.side_join);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    for (auto& e : h->ev) if (e) cudaEventDestroy(e);
    if (h->rb) cudaFreeHost(h->rb);
    if (h->d.norm_host) cudaFreeHost(h->d.norm_host);
    cudaGetLastError();
    delete h;
    return ITOKMC_OK;
}

int itokmc_set_particles(itokmc_handle* h, const double* x, const double* y, const double* z, const uint32_t* w,
                         const int32_t* realization, int64_t n, int32_t mem)
{
    return itokmc_set_particles_species(h, x, y, z, w, realization, nullptr, n, mem);
}

int itokmc_set_particles_species(itokmc_handle* h, const double* x, const double* y, const double* z,
                                 const uint32_t* w, const int32_t* realization, const int32_t* species, int64_t n,
                                 int32_t mem)
{
    IK_GUARD(h);
    h->stage = 0;
    if (n < 0 || (n > 0 && (!x || !y || !z || !w))) return fail(h, ITOKMC_ERR_ARG, "bad particle arrays");
    if (n > (int64_t)h->cap) return fail(h, ITOKMC_ERR_CAPACITY, "more particles than particle_capacity");
    if (h->P.R > 1 && n > 0 && !realization) return fail(h, ITOKMC_ERR_ARG, "realization array required when R > 1");
    // stage the SoA arrays in scratch: the (about to be overwritten) record
    // buffer A of the FP64 form, the merge work buffer of the mixed form
    unsigned char* st = h->d.mixed ? h->d.work : reinterpret_cast<unsigned char*>(h->d.recA);
    double* dx = reinterpret_cast<double*>(st);
    double* dy = dx + n;
    double* dz = dy + n;
    uint32_t* dw = reinterpret_cast<uint32_t*>(dz + n);
    int32_t* dr = realization ? reinterpret_cast<int32_t*>(dw + n) : nullptr;
    const cudaMemcpyKind k = mem == ITOKMC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (n > 0) {
        IK_CHECK(h, cudaMemcpyAsync(dx, x, n * sizeof(double), k, h->s));
        IK_CHECK(h, cudaMemcpyAsync(dy, y, n * sizeof(double), k, h->s));
        IK_CHECK(h, cudaMemcpyAsync(dz, z, n * sizeof(double), k, h->s));
        IK_CHECK(h, cudaMemcpyAsync(dw, w, n * sizeof(uint32_t), k, h->s));
        if (dr) IK_CHECK(h, cudaMemcpyAsync(dr, realization, n * sizeof(int32_t), k, h->s));
    }
    // the species (mobile ions) in the push keys' buffer, free until the next push
    int32_t* dsp = (species && n > 0) ? reinterpret_cast<int32_t*>(h->d.keyB) : nullptr;
    if (dsp) IK_CHECK(h, cudaMemcpyAsync(dsp, species, n * sizeof(int32_t), k, h->s));
    ik::launch_set_particles(h->P, h->d, dx, dy, dz, dw, dr, dsp, (uint32_t)n, h->Gp, h->s);
    int rc = readback(h);
    if (rc) return rc;
    if (h->rb->ctr.err) {
        h->N = 0;
        cudaMemsetAsync(h->d.cell_start, 0, (h->Gp + 1) * sizeof(uint32_t), h->s);
        cudaStreamSynchronize(h->s);
        return fail(h, ITOKMC_ERR_ARG, "particle outside the domain, zero weight, bad realization or species");
    }
    h->N = (uint32_t)n;
    h->st.n_particles = n;
    return ITOKMC_OK;
}

int itokmc_read_particles(itokmc_handle* h, double* x, double* y, double* z, uint32_t* w, int32_t* realization,
                          int64_t* cell, int64_t cap, int64_t* n_out, int32_t mem)
{
    IK_GUARD(h);
    if (mem != ITOKMC_HOST) return fail(h, ITOKMC_ERR_ARG, "read_particles copies to host memory");
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    const uint32_t N = h->N;
    if (n_out) *n_out = N;
    if ((int64_t)N > cap) return fail(h, ITOKMC_ERR_CAPACITY, "output buffer smaller than the particle count");
    const uint32_t n3 = (uint32_t)h->P.n3;
    if (!h->d.mixed) {
        std::vector<ik::P64> buf(N);
        if (N) IK_CHECK(h, cudaMemcpyAsync(buf.data(), h->d.recA, N * sizeof(ik::P64), cudaMemcpyDeviceToHost, h->s));
        IK_CHECK(h, cudaStreamSynchronize(h->s));
        for (uint32_t i = 0; i < N; ++i) {
            if (x) x[i] = buf[i].x;
            if (y) y[i] = buf[i].y;
            if (z) z[i] = buf[i].z;
            if (w) w[i] = buf[i].w;
            if (realization) realization[i] = (int32_t)(buf[i].cell / n3);
            if (cell) cell[i] = (int64_t)(buf[i].cell % n3);
        }
        return ITOKMC_OK;
    }
    // mixed form: absolute position lo + (i + offset) h
    std::vector<ik::P32> buf(N);
    std::vector<uint32_t> cb(N);
    if (N) {
        IK_CHECK(h, cudaMemcpyAsync(buf.data(), h->d.rA32, N * sizeof(ik::P32), cudaMemcpyDeviceToHost, h->s));
        IK_CHECK(h, cudaMemcpyAsync(cb.data(), h->d.cellA32, N * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->s));
    }
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    const uint32_t n = (uint32_t)h->P.n;
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t c = cb[i] % n3;
        const uint32_t id[3] = { c % n, (c / n) % n, c / (n * n) };
        const float o[3] = { buf[i].ox, buf[i].oy, buf[i].oz };
        double X[3];
        for (int a = 0; a < 3; ++a) X[a] = h->P.lo[a] + ((double)id[a] + (double)o[a]) * h->P.h[a];
        if (x) x[i] = X[0];
        if (y) y[i] = X[1];
        if (z) z[i] = X[2];
        if (w) w[i] = buf[i].w;
        if (realization) realization[i] = (int32_t)(cb[i] / n3);
        if (cell) cell[i] = (int64_t)c;
    }
    return ITOKMC_OK;
}

int itokmc_set_ions(itokmc_handle* h, const int64_t* npos, const int64_t* nneg, int32_t mem)
{
    IK_GUARD(h);
    if (h->P.S != 1)
        return fail(h, ITOKMC_ERR_ARG, "mobile ions are particles: set them with itokmc_set_particles_species");
    const cudaMemcpyKind k = mem == ITOKMC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (npos) IK_CHECK(h, cudaMemcpyAsync(h->d.Npos, npos, h->G * sizeof(int64_t), k, h->s));
    if (nneg) IK_CHECK(h, cudaMemcpyAsync(h->d.Nneg, nneg, h->G * sizeof(int64_t), k, h->s));
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    return ITOKMC_OK;
}

int itokmc_set_field(itokmc_handle* h, const double* E, int32_t mem)
{
    IK_GUARD(h);
    if (!E) return fail(h, ITOKMC_ERR_ARG, "NULL field");
    const cudaMemcpyKind k = mem == ITOKMC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    IK_CHECK(h, cudaMemcpyAsync(h->d.stage, E, 3 * h->G * sizeof(double), k, h->s));
    ik::launch_pack_field(h->P, h->d, h->d.stage, h->s);
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    return cuda_check(h, cudaGetLastError(), "set_field");
}

int itokmc_solve_field(itokmc_handle* h)
{
    IK_GUARD(h);
    cudaMemsetAsync(h->d.ctr, 0, sizeof(ik::Counters), h->s);
    ik::launch_deposit_only(h->P, h->d, h->N, h->s);
    ik::launch_rho(h->P, h->d, h->G, h->s);
    int rc = readback(h);
    if (rc) return rc;
    rc = status_of_err(h, h->rb->ctr.err);
    if (rc) return rc;
    return stage_field(h);
}

int itokmc_run_stage(itokmc_handle* h, int32_t stage)
{
    IK_GUARD(h);
    switch (stage) {
    case ITOKMC_STAGE_TRANSPORT: return stage_transport(h);
    case ITOKMC_STAGE_KMC: {
        int rc = stage_kmc(h);
        if (rc) return rc;
        IK_CHECK(h, cudaMemcpyAsync(&h->rb->ctr, h->d.ctr, sizeof(ik::Counters), cudaMemcpyDeviceToHost, h->s));
        IK_CHECK(h, cudaStreamSynchronize(h->s));
        return status_of_err(h, h->rb->ctr.err & ik::DERR_KMC);
    }
    case ITOKMC_STAGE_PARTICLES: return stage_particles(h);
    case ITOKMC_STAGE_FIELD: return stage_field(h);
    default: return fail(h, ITOKMC_ERR_ARG, "unknown stage");
    }
}

int itokmc_transport_semi_implicit(itokmc_handle* h, int32_t* cycles_out, double* rel_out)
{
    IK_GUARD(h);
    return stage_semi_transport(h, cycles_out, rel_out);
}

int itokmc_autotune(itokmc_handle* h, itokmc_tuning* out)
{
    IK_GUARD(h);
    ik::Dev& d = h->d;
    const size_t cells = h->G;
    double* phi0 = d.lev[0].phi;
    // the stage buffer (3 G doubles) holds the initial potential
    IK_CHECK(h, cudaMemcpyAsync(d.stage, phi0, cells * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    const int F0 = d.phi_F;
    itokmc_tuning t{};
    int best = -1;
    double best_ms = 0.0;
    int best_cyc = 0;
    const int prec = d.phi_F > 0 ? 2 : h->field_prec;
    for (int a = 1; a <= 3; ++a)
        for (int b = 1; b <= 3; ++b) {
            const int k = t.n_tried++;
            t.nu_tried[k][0] = a;
            t.nu_tried[k][1] = b;
            double ms = -1.0;
            int cyc = 0;
            for (int rep = 0; rep < 2; ++rep) {
                // from a zero potential: a solve that needs many cycles ranks
                // the pairs by their convergence per unit time
                IK_CHECK(h, cudaMemsetAsync(phi0, 0, cells * sizeof(double), h->s));
                d.phi_F = F0;
                double rel = 0.0;
                IK_CHECK(h, cudaEventRecord(h->ev[6], h->s));
                const int st = ik::field_solve(h->P, d, prec, h->cfg.mg_rtol, a, b, h->rb->ctr.rho_absmax,
                                               h->cfg.mg_max_cycles, h->s, &cyc, &rel);
                IK_CHECK(h, cudaEventRecord(h->ev[7], h->s));
                IK_CHECK(h, cudaStreamSynchronize(h->s));
                if (st == -3) return cuda_check(h, cudaGetLastError(), "autotune field solve");
                if (st != 0) { ms = -1.0; break; }
                const double m = elapsed(h, 6, 7);
                ms = ms < 0.0 ? m : std::min(ms, m);
            }
            t.ms_tried[k] = ms;
            if (ms >= 0.0 && (best < 0 || ms < best_ms)) {
                best = k;
                best_ms = ms;
                best_cyc = cyc;
            }
        }
    // restore the potential and the field of the initial state
    IK_CHECK(h, cudaMemcpyAsync(phi0, d.stage, cells * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    d.phi_F = F0;
    ik::launch_efield(h->P, d, h->s);
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    if (best < 0) return fail(h, ITOKMC_ERR_NOCONV, "autotune: no smoother pair converged");
    h->cfg.mg_nu1 = t.nu_tried[best][0];
    h->cfg.mg_nu2 = t.nu_tried[best][1];
    t.mg_nu1 = h->cfg.mg_nu1;
    t.mg_nu2 = h->cfg.mg_nu2;
    t.ms_field = best_ms;
    t.cycles = best_cyc;
    // the push's deposit window: trial pushes of the current particles; the
    // last deposit (ne_fix, X) is kept in the merge work area meanwhile
    t.dep_win = h->P.dep_win;
    t.n_dep_tried = 0;
    const size_t dep_bytes = h->Gp * sizeof(unsigned long long);
    if (h->N > 0 && d.work_bytes >= 3 * dep_bytes + 16) {
        IK_CHECK(h, cudaMemcpyAsync(d.work, d.ne_fix, dep_bytes, cudaMemcpyDeviceToDevice, h->s));
        IK_CHECK(h, cudaMemcpyAsync(d.work + dep_bytes, d.Xe, dep_bytes, cudaMemcpyDeviceToDevice, h->s));
        // every trial's deposit must equal the first one's (integer sums)
        unsigned long long* first = reinterpret_cast<unsigned long long*>(d.work + 2 * dep_bytes);
        unsigned int* differs = reinterpret_cast<unsigned int*>(d.work + 3 * dep_bytes);
        IK_CHECK(h, cudaMemsetAsync(differs, 0, sizeof(unsigned int), h->s));
        const int cand[ITOKMC_TUNE_DEPOSIT] = { 0, 256, 512, 1024, ik::DEP_WIN_MAX };
        float best_push = -1.f;
        int best_win = h->P.dep_win;
        for (int k = 0; k < ITOKMC_TUNE_DEPOSIT; ++k) {
            h->P.dep_win = cand[k];
            const float ms = ik::time_push(h->P, d, h->N, h->s, 3);
            if (k == 0) IK_CHECK(h, cudaMemcpyAsync(first, d.ne_fix, dep_bytes, cudaMemcpyDeviceToDevice, h->s));
            else ik::launch_diff_flag(first, d.ne_fix, h->Gp, differs, h->s);
            t.dep_tried[k] = cand[k];
            t.ms_dep_tried[k] = ms;
            ++t.n_dep_tried;
            if (ms >= 0.f && (best_push < 0.f || ms < best_push)) { best_push = ms; best_win = cand[k]; }
        }
        h->P.dep_win = best_win;
        t.dep_win = best_win;
        unsigned int diff = 0;
        IK_CHECK(h, cudaMemcpyAsync(&diff, differs, sizeof diff, cudaMemcpyDeviceToHost, h->s));
        IK_CHECK(h, cudaMemcpyAsync(d.ne_fix, d.work, dep_bytes, cudaMemcpyDeviceToDevice, h->s));
        IK_CHECK(h, cudaMemcpyAsync(d.Xe, d.work + dep_bytes, dep_bytes, cudaMemcpyDeviceToDevice, h->s));
        IK_CHECK(h, cudaStreamSynchronize(h->s));
        drop_graphs(h);                      // the kernels' parameters changed
        if (diff) return fail(h, ITOKMC_ERR_INTERNAL, "autotune: deposit windows gave different densities");
    }
    if (out) *out = t;
    return cuda_check(h, cudaGetLastError(), "autotune");
}

int itokmc_advance_counter(itokmc_handle* h)
{
    IK_GUARD(h);
    h->step += 1;
    h->P.step = (uint32_t)h->step;
    h->st.step = h->step;
    return ITOKMC_OK;
}

int itokmc_step(itokmc_handle* h, int32_t nsteps)
{
    IK_GUARD(h);
    if (nsteps < 0) return fail(h, ITOKMC_ERR_ARG, "nsteps < 0");
    for (int k = 0; k < nsteps; ++k) {
        int rc = h->cfg.dt_adapt ? choose_step(h) : ITOKMC_OK;
        if (!rc) rc = h->cfg.coupling == ITOKMC_SEMI_IMPLICIT ? semi_step(h)
                                                                : (graph_eligible(h) ? graph_step(h) : full_step(h));
        if (rc) return rc;
        ++h->steps_done;
        itokmc_advance_counter(h);
    }
    h->st.n_particles = h->N;
    return ITOKMC_OK;
}

int itokmc_read_densities(itokmc_handle* h, int32_t r, int32_t which, void* host_out, size_t bytes)
{
    IK_GUARD(h);
    if (!host_out) return fail(h, ITOKMC_ERR_ARG, "NULL output");
    if (r < -1 || r >= h->P.R) return fail(h, ITOKMC_ERR_ARG, "realization out of range");
    const size_t n3 = (size_t)h->P.n3;
    const size_t cnt = r < 0 ? h->G : n3;
    const size_t off = r < 0 ? 0 : (size_t)r * n3;
    const void* src = nullptr;
    int blocks = 1;
    switch (which) {
    case ITOKMC_NE_FIX: src = h->d.ne_fix; break;
    case ITOKMC_XE: src = h->d.Xe; break;
    // mobile ions: the NGP counts of the ion blocks' last deposit
    case ITOKMC_NPOS: src = h->P.S == 3 ? static_cast<const void*>(h->d.Xe + h->G) : h->d.Npos; break;
    case ITOKMC_NNEG: src = h->P.S == 3 ? static_cast<const void*>(h->d.Xe + 2 * h->G) : h->d.Nneg; break;
    case ITOKMC_PHI:
        if (h->d.phi_F > 0) {
            ik::launch_phi_to_double(h->P, h->d, h->d.stage, h->s);
            src = h->d.stage;
        } else {
            src = h->d.lev[0].phi;
        }
        break;
    case ITOKMC_RHO: src = h->d.rho; break;
    case ITOKMC_E:
        ik::launch_unpack_field(h->P, h->d, h->d.stage, h->s);
        src = h->d.stage; blocks = 3; break;
    case ITOKMC_FIRINGS: src = h->d.fired; blocks = 5; break;
    default: return fail(h, ITOKMC_ERR_ARG, "unknown field");
    }
    if (bytes < blocks * cnt * 8) return fail(h, ITOKMC_ERR_ARG, "output buffer too small");
    for (int b = 0; b < blocks; ++b)
        IK_CHECK(h, cudaMemcpyAsync(static_cast<char*>(host_out) + b * cnt * 8,
                                    static_cast<const char*>(src) + (b * h->G + off) * 8, cnt * 8,
                                    cudaMemcpyDeviceToHost, h->s));
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    return cuda_check(h, cudaGetLastError(), "read_densities");
}

int itokmc_get_stats(itokmc_handle* h, itokmc_stats* st)
{
    IK_GUARD(h);
    if (!st) return ITOKMC_ERR_ARG;
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    h->st.n_particles = h->N;
    h->st.step = h->step;
    h->st.kernel_launches = (int64_t)ik::g_launches;
    *st = h->st;
    return ITOKMC_OK;
}

int itokmc_num_particles(itokmc_handle* h, int64_t* n_out)
{
    IK_GUARD(h);
    if (!n_out) return ITOKMC_ERR_ARG;
    IK_CHECK(h, cudaStreamSynchronize(h->s));
    *n_out = h->N;
    return ITOKMC_OK;
}

int itokmc_kmc0d(const itokmc_config* cfg, double E_mag, int64_t X0, int32_t n_real, int32_t n_steps, int64_t* X,
                 int32_t mem)
{
    if (!cfg || !X) return fail(nullptr, ITOKMC_ERR_ARG, "kmc0d: NULL argument");
    if (n_real < 1 || n_steps < 0 || X0 < 0 || !(E_mag >= 0.0) || !(cfg->dt > 0.0) || cfg->mu < 0.0 ||
        cfg->n_ssa < 1 || cfg->n_crit < 0 || (mem != ITOKMC_HOST && mem != ITOKMC_DEVICE))
        return fail(nullptr, ITOKMC_ERR_ARG, "kmc0d: n_real >= 1, n_steps >= 0, X0 >= 0, E >= 0, dt > 0, mu >= 0");
    if (cfg->precision != ITOKMC_FP64 && cfg->precision != ITOKMC_MIXED)
        return fail(nullptr, ITOKMC_ERR_ARG, "kmc0d: precision");
    itokmc_config c = *cfg;
    c.n[0] = c.n[1] = c.n[2] = 8;                      // no grid: any valid size for the parameters
    for (int a = 0; a < 3; ++a) { c.lo[a] = 0.0; c.hi[a] = 1.0; }
    c.n_realizations = 1;
    ik::Params P{};
    fill_params(&c, P);
    cudaStream_t s = (cudaStream_t)cfg->stream;
    const size_t bytes = (size_t)n_real * (size_t)(n_steps + 1) * sizeof(long long);
    long long* dX = reinterpret_cast<long long*>(X);
    ik::Counters* ctr = nullptr;
    bool own = false;
    if (cudaMalloc(reinterpret_cast<void**>(&ctr), sizeof(ik::Counters)) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, ITOKMC_ERR_OOM, "kmc0d: counters");
    }
    if (mem == ITOKMC_HOST) {
        if (cudaMalloc(reinterpret_cast<void**>(&dX), bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ctr);
            return fail(nullptr, ITOKMC_ERR_OOM, "kmc0d: trajectories");
        }
        own = true;
    }
    cudaMemsetAsync(ctr, 0, sizeof(ik::Counters), s);
    ik::launch_kmc0d(P, cfg->precision == ITOKMC_MIXED, E_mag, (long long)X0, (uint32_t)n_real, n_steps, dX, ctr, s);
    unsigned err = 0;
    cudaMemcpyAsync(&err, &ctr->err, sizeof err, cudaMemcpyDeviceToHost, s);
    if (own) cudaMemcpyAsync(X, dX, bytes, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (own) cudaFree(dX);
    cudaFree(ctr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, ITOKMC_ERR_CUDA, std::string("kmc0d: ") + cudaGetErrorString(e));
    }
    if (err) return fail(nullptr, ITOKMC_ERR_KMC, "kmc0d: KMC iteration guard hit");
    return ITOKMC_OK;
}

const char* itokmc_last_error(const itokmc_handle* h) { return h ? h->err.c_str() : ik::g_noh_err; }

const char* itokmc_version(void) { return "itokmc 0.1 (sm_103a)"; }

}  // extern "C"
