// ik_checkpoint.cu -- checkpoint files of a run (itokmc_save / itokmc_load).
//
// A checkpoint holds everything the next step reads, so that a run resumed
// from it continues bit for bit as the uninterrupted run would (every random
// draw is a Philox counter of (seed, index, step, tag), so the step counter
// and the canonical particle order fix the draws): the configuration it was
// written for, the step counter and the smoother counts in use, the particles
// in canonical order with the per-cell offsets, the ion counts, the field of
// the next step, the potential and the previous potential (the initial guess
// of the next solve is extrapolated from both), the fixed-point exponent of
// the mixed potential, and the mesh densities of the last deposit.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/itokmc.h"
#include "ik_handle.h"


namespace {

constexpr char MAGIC[8] = { 'I', 'T', 'O', 'K', 'M', 'C', 'K', '3' };

// The part of the configuration a checkpoint is bound to (the physics, the
// grid and the form; not the allocator, the stream or the capacity).
struct CkptHeader {
    char magic[8];
    int32_t n, R, precision, field_prec, frac_bits, ppc, n_new, n_crit, n_ssa, pad0;
    double lo[3], hi[3], dt, mu, D, alpha_A, alpha_B, eta, E0, photon_ratio, kappa_lo, kappa_hi, eps, mg_rtol;
    uint64_t seed0;
    int64_t step;
    int32_t mg_nu1, mg_nu2, phi_F, have_prev;
    uint32_t N, pad1;
    uint64_t G;
    double beta_ep, beta_np;
    int32_t mobile_ions, pad2;
    double mu_ion, D_ion;
};

CkptHeader header_of(const ik::HandleView& v)
{
    CkptHeader H;
    std::memset(&H, 0, sizeof H);
    std::memcpy(H.magic, MAGIC, 8);
    const itokmc_config& c = *v.cfg;
    H.n = c.n[0]; H.R = c.n_realizations; H.precision = c.precision; H.field_prec = v.field_prec;
    H.frac_bits = c.frac_bits; H.ppc = c.ppc; H.n_new = c.n_new; H.n_crit = c.n_crit; H.n_ssa = c.n_ssa;
    for (int a = 0; a < 3; ++a) { H.lo[a] = c.lo[a]; H.hi[a] = c.hi[a]; }
    H.dt = c.dt; H.mu = c.mu; H.D = c.D; H.alpha_A = c.alpha_A; H.alpha_B = c.alpha_B; H.eta = c.eta; H.E0 = c.E0;
    H.photon_ratio = c.photon_ratio; H.kappa_lo = c.kappa_lo; H.kappa_hi = c.kappa_hi; H.eps = c.eps;
    H.mg_rtol = c.mg_rtol; H.seed0 = c.seed0;
    H.step = *v.step;
    H.mg_nu1 = c.mg_nu1; H.mg_nu2 = c.mg_nu2;
    H.phi_F = v.d->phi_F; H.have_prev = v.d->have_prev ? 1 : 0;
    H.N = *v.N;
    H.G = v.G;
    H.beta_ep = c.beta_ep; H.beta_np = c.beta_np;
    H.mobile_ions = c.mobile_ions; H.mu_ion = c.mu_ion; H.D_ion = c.D_ion;
    return H;
}

// The first configuration field in which two headers differ ("" if none).
const char* mismatch(const CkptHeader& a, const CkptHeader& b)
{
#define IK_SAME(f) if (std::memcmp(&a.f, &b.f, sizeof a.f) != 0) return #f
    IK_SAME(n); IK_SAME(R); IK_SAME(precision); IK_SAME(field_prec); IK_SAME(frac_bits); IK_SAME(ppc);
    IK_SAME(n_new); IK_SAME(n_crit); IK_SAME(n_ssa); IK_SAME(lo); IK_SAME(hi); IK_SAME(dt); IK_SAME(mu);
    IK_SAME(D); IK_SAME(alpha_A); IK_SAME(alpha_B); IK_SAME(eta); IK_SAME(E0); IK_SAME(photon_ratio);
    IK_SAME(kappa_lo); IK_SAME(kappa_hi); IK_SAME(eps); IK_SAME(mg_rtol); IK_SAME(seed0); IK_SAME(G);
    IK_SAME(beta_ep); IK_SAME(beta_np); IK_SAME(mobile_ions); IK_SAME(mu_ion); IK_SAME(D_ion);
#undef IK_SAME
    return "";
}

// The device arrays of a checkpoint, in file order, with their sizes.
struct Blob {
    void* p;
    size_t bytes;
};

std::vector<Blob> blobs_of(const ik::HandleView& v, uint32_t N)
{
    ik::Dev& d = *v.d;
    const size_t G = v.G, Gp = v.Gp;
    std::vector<Blob> b;
    if (d.mixed) {
        b.push_back({ d.rA32, (size_t)N * sizeof(ik::P32) });
        b.push_back({ d.cellA32, (size_t)N * sizeof(uint32_t) });
        b.push_back({ d.E32, G * sizeof(float4) });
    } else {
        b.push_back({ d.recA, (size_t)N * sizeof(ik::P64) });
        b.push_back({ d.E, G * sizeof(ik::E64) });
    }
    b.push_back({ d.cell_start, (Gp + 1) * sizeof(uint32_t) });
    b.push_back({ d.Npos, G * sizeof(int64_t) });
    b.push_back({ d.Nneg, G * sizeof(int64_t) });
    b.push_back({ d.lev[0].phi, G * sizeof(double) });     // FP64 potential, or the int64 fixed-point one
    b.push_back({ d.phi_prev, G * sizeof(double) });
    b.push_back({ d.ne_fix, Gp * sizeof(unsigned long long) });
    b.push_back({ d.Xe, Gp * sizeof(unsigned long long) });
    b.push_back({ d.rho, G * sizeof(int64_t) });
    b.push_back({ d.fired, 5 * G * sizeof(int64_t) });
    b.push_back({ d.gain, Gp * sizeof(int64_t) });
    return b;
}

constexpr size_t CHUNK = 64u << 20;

}  // namespace

extern "C" int itokmc_save(itokmc_handle* h, const char* path)
{
    ik::HandleView v;
    int rc = ik::handle_view(h, &v);
    if (rc) return rc;
    if (!path) return ik::handle_fail(h, ITOKMC_ERR_ARG, "save: NULL path");
    if (cudaStreamSynchronize(v.s) != cudaSuccess) return ik::handle_fail(h, ITOKMC_ERR_CUDA, "save: stream");
    const CkptHeader H = header_of(v);
    FILE* f = std::fopen(path, "wb");
    if (!f) return ik::handle_fail(h, ITOKMC_ERR_ARG, (std::string("save: cannot open ") + path).c_str());
    bool ok = std::fwrite(&H, sizeof H, 1, f) == 1;
    std::vector<unsigned char> buf;
    for (const Blob& b : blobs_of(v, H.N)) {
        for (size_t o = 0; ok && o < b.bytes; o += CHUNK) {
            const size_t m = b.bytes - o < CHUNK ? b.bytes - o : CHUNK;
            buf.resize(m);
            if (cudaMemcpy(buf.data(), static_cast<unsigned char*>(b.p) + o, m, cudaMemcpyDeviceToHost) != cudaSuccess) {
                std::fclose(f);
                return ik::handle_fail(h, ITOKMC_ERR_CUDA, "save: device copy");
            }
            ok = std::fwrite(buf.data(), 1, m, f) == m;
        }
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return ik::handle_fail(h, ITOKMC_ERR_ARG, "save: write failed");
    return ITOKMC_OK;
}

extern "C" int itokmc_load(itokmc_handle* h, const char* path)
{
    ik::HandleView v;
    int rc = ik::handle_view(h, &v);
    if (rc) return rc;
    *v.stage = 0;                                 // a checkpoint is a step boundary
    if (!path) return ik::handle_fail(h, ITOKMC_ERR_ARG, "load: NULL path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return ik::handle_fail(h, ITOKMC_ERR_ARG, (std::string("load: cannot open ") + path).c_str());
    CkptHeader F;
    if (std::fread(&F, sizeof F, 1, f) != 1 || std::memcmp(F.magic, MAGIC, 8) != 0) {
        std::fclose(f);
        return ik::handle_fail(h, ITOKMC_ERR_ARG, "load: not an itokmc checkpoint");
    }
    const CkptHeader mine = header_of(v);
    const char* m = mismatch(F, mine);
    if (*m) {
        std::fclose(f);
        return ik::handle_fail(h, ITOKMC_ERR_ARG,
                                   (std::string("load: checkpoint of another configuration (") + m + ")").c_str());
    }
    if (F.N > v.cap) {
        std::fclose(f);
        return ik::handle_fail(h, ITOKMC_ERR_CAPACITY, "load: more particles than particle_capacity");
    }
    if (cudaStreamSynchronize(v.s) != cudaSuccess) {
        std::fclose(f);
        return ik::handle_fail(h, ITOKMC_ERR_CUDA, "load: stream");
    }
    std::vector<unsigned char> buf;
    bool ok = true;
    for (const Blob& b : blobs_of(v, F.N)) {
        for (size_t o = 0; ok && o < b.bytes; o += CHUNK) {
            const size_t mm = b.bytes - o < CHUNK ? b.bytes - o : CHUNK;
            buf.resize(mm);
            ok = std::fread(buf.data(), 1, mm, f) == mm;
            if (ok && cudaMemcpy(static_cast<unsigned char*>(b.p) + o, buf.data(), mm, cudaMemcpyHostToDevice) != cudaSuccess) {
                std::fclose(f);
                return ik::handle_fail(h, ITOKMC_ERR_CUDA, "load: device copy");
            }
        }
    }
    std::fclose(f);
    if (!ok) return ik::handle_fail(h, ITOKMC_ERR_ARG, "load: truncated checkpoint");
    *v.N = F.N;
    *v.step = F.step;
    v.P->step = (uint32_t)F.step;
    v.cfg->mg_nu1 = F.mg_nu1;
    v.cfg->mg_nu2 = F.mg_nu2;
    v.d->phi_F = F.phi_F;
    v.d->have_prev = F.have_prev != 0;
    return ITOKMC_OK;
}
