// ldpm_api.cu -- host runtime behind the C ABI of include/ldpm.h.
//
// Set-up (ldpm_create): validation of the mesh rules, facet frames/arms/projected areas
// (paper Sec. 2), lumped mass (Sec. 3.2.5), Morton ordering of particles and tetrahedra, the
// particle-to-facet-end CSR list in a fixed order, upload, and the critical-step estimate.
// Stepping (ldpm_step): the kernels of ldpm_kernels.cu, replayed from captured CUDA graphs.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ldpm.h"
#include "ldpm_internal.h"

using namespace ldpm;

namespace {
thread_local std::string g_err;
}  // namespace

void ldpm::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

namespace {

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(e_ == cudaErrorMemoryAllocation ? LDPM_E_OOM : LDPM_E_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    } while (0)

constexpr int kTile = 32;  // tetrahedra per facet-pass block (padding granularity)
constexpr int kEdgeA[6] = {0, 0, 0, 1, 1, 2};
constexpr int kEdgeB[6] = {1, 2, 3, 2, 3, 3};

int edge_of(int a, int b)
{
    if (a > b) std::swap(a, b);
    for (int e = 0; e < 6; ++e)
        if (kEdgeA[e] == a && kEdgeB[e] == b) return e;
    return -1;
}

uint32_t spread10(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

uint32_t morton3(const double *p, const double *lo, const double *span)
{
    uint32_t c[3];
    for (int a = 0; a < 3; ++a) {
        double t = span[a] > 0 ? (p[a] - lo[a]) / span[a] : 0.0;
        t = std::min(std::max(t, 0.0), 1.0);
        c[a] = (uint32_t)std::min(1023.0, std::floor(t * 1024.0));
    }
    return spread10(c[0]) | (spread10(c[1]) << 1) | (spread10(c[2]) << 2);
}

// fn(lo, hi) over contiguous chunks of [0, n) on up to 16 host threads (one thread below 65536
// items); returns the smallest of the chunks' results.  The checks below return the first failing
// item of their chunk (or a sentinel), so the result is the item a sequential loop would report.
// Host threads parallel_min uses for n items: up to 16, one below 65536 items.
unsigned host_threads(int64_t n)
{
    const unsigned hw = std::thread::hardware_concurrency();
    return n < 65536 ? 1u : std::max(1u, std::min(hw, 16u));
}

template <class Fn>
int64_t parallel_min(int64_t n, Fn &&fn)
{
    const unsigned nt = host_threads(n);
    if (nt == 1) return fn((int64_t)0, n);
    std::vector<int64_t> res(nt, INT64_MAX);
    std::vector<std::thread> th;
    const int64_t chunk = (n + nt - 1) / nt;
    try {
        for (unsigned i = 0; i < nt; ++i) {
            const int64_t lo = std::min(n, (int64_t)i * chunk), hi = std::min(n, lo + chunk);
            th.emplace_back([&, i, lo, hi]() { res[i] = fn(lo, hi); });
        }
    } catch (...) {  // no thread could be started: finish on this one
        for (auto &t : th) t.join();
        return fn((int64_t)0, n);
    }
    for (auto &t : th) t.join();
    return *std::min_element(res.begin(), res.end());
}

// Stable order of n items by 32-bit key (ties by index): LSD radix sort of (key, index) pairs, 8 bits
// per pass.
std::vector<int32_t> order_by_key(const std::vector<uint32_t> &key)
{
    const size_t n = key.size();
    std::vector<uint32_t> ka(key), kb(n);
    std::vector<int32_t> ia(n), ib(n);
    std::iota(ia.begin(), ia.end(), 0);
    for (int sh = 0; sh < 32; sh += 8) {
        size_t cnt[257] = {0};
        for (size_t i = 0; i < n; ++i) ++cnt[((ka[i] >> sh) & 0xffu) + 1];
        if (cnt[((ka.empty() ? 0 : ka[0]) >> sh & 0xffu) + 1] == n) continue;  // one digit value: order kept
        for (int d = 0; d < 256; ++d) cnt[d + 1] += cnt[d];
        for (size_t i = 0; i < n; ++i) {
            const size_t pos = cnt[(ka[i] >> sh) & 0xffu]++;
            kb[pos] = ka[i];
            ib[pos] = ia[i];
        }
        ka.swap(kb);
        ia.swap(ib);
    }
    return ia;
}

template <class R>
void law_const(const ldpm_material &mt, double dt, LawConst<R> &c)
{
    const double E0 = mt.E0, a = mt.alpha;
    c.E0 = R(E0);
    c.alpha = R(a);
    c.inv_alpha = R(1.0 / a);
    c.sigma_t = R(mt.sigma_t);
    c.four_alpha_over_r2 = R(4.0 * a / (mt.r_st * mt.r_st));
    c.Hs_over_alpha = R(mt.r_s * E0 / a);
    c.n_t = R(mt.n_t);
    c.l_t = R(mt.l_t);
    c.sigma_c0 = R(mt.sigma_c0);
    c.Hc0 = R(mt.Hc0_E0 * E0);
    c.Hc1 = R(mt.Hc1_E0 * E0);
    c.kc1 = R(mt.kc1);
    c.kc2 = R(mt.kc2);
    c.ec0 = R(mt.sigma_c0 / E0);
    c.ec1 = R(mt.kc0 * mt.sigma_c0 / E0);
    c.eV0 = R(mt.kc3 * mt.sigma_c0 / E0);
    c.beta = R(mt.beta);
    c.Ed = R(mt.Ed_E0 * E0);
    c.mu_diff_sN0 = R((mt.mu0 - mt.mu_inf) * mt.sigma_N0);
    c.mu_inf = R(mt.mu_inf);
    c.inv_sigma_N0 = R(1.0 / mt.sigma_N0);
    c.sigma_s = R(mt.r_st * mt.sigma_t);
    c.dt = R(dt);
    // FP32: squares of strains below ~1e-19 underflow; 1e-15 keeps every product of the law normal
    // and changes tractions by < E0 * 1e-15.  FP64: the oracle's threshold.
    c.tiny_strain = R(sizeof(R) == 4 ? 1e-15 : 1e-150);
    c.four_over_r2 = R(4.0 / (mt.r_st * mt.r_st));
    c.r_st = R(mt.r_st);
    c.Hc0_E0 = R(mt.Hc0_E0);
    c.Hc1_E0 = R(mt.Hc1_E0);
    c.kc0 = R(mt.kc0);
    c.kc3 = R(mt.kc3);
    c.Ed_E0 = R(mt.Ed_E0);
    c.r_s = R(mt.r_s);
    c.k_t = R(mt.k_t);
    c.elastic = mt.elastic;
}

struct SpecHost {
    int32_t N = 0, T = 0, F = 0;  // caller sizes
    int32_t p0 = 0, t0 = 0;        // internal offsets (t0 multiple of kTile)
    int32_t T_pad = 0;
    ldpm_material mat{};
    double dt = 0, ramp_time = 0, W_kin0 = 0;
    std::vector<int32_t> perm_p;  // internal rank -> caller particle
    std::vector<int32_t> inv_p;   // caller particle -> internal rank
    std::vector<int64_t> fmap;    // caller facet -> internal facet (global index)
    std::vector<int32_t> tmap;    // caller tetrahedron -> internal tetrahedron (global index)
    std::vector<uint8_t> fswap;   // caller facet I is the internal b vertex
};

}  // namespace

struct ldpm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int prec = LDPM_FP64;
    int graph_chunk = 32;
    DeviceModel dm;
    std::vector<SpecHost> sp;
    std::vector<double> x_int;     // [N][3] internal order
    std::vector<double> inv_mass;  // [N][6]
    std::vector<double> pconst_h;  // [N][8]
    double *d_partial = nullptr, *d_out16 = nullptr, *h_out16 = nullptr;
    unsigned *d_ticket = nullptr;       // block counter of the energy reduction
    int32_t *d_umap = nullptr;          // caller's facets of all specimens, concatenated: 2 f + orientation flip
    int32_t *d_pmap = nullptr;          // caller's particles of all specimens, concatenated: internal particle
    std::vector<int64_t> ufoff;         // [n_spec + 1] offsets of each specimen's facets in d_umap
    double *d_scratch = nullptr;        // state read-back scratch, grown on demand
    size_t scratch_n = 0;
    std::map<int64_t, cudaGraphExec_t> graphs;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::array<int, 3>> ev_pairs;  // (kernel id, event index of start, event index of end)
    double prof_ms[6] = {0, 0, 0, 0, 0, 0};  // kick, facet pass, particle pass, reverse facet, reverse particle,
    int64_t prof_cnt[6] = {0, 0, 0, 0, 0, 0};  // persistent step launch
    int launch_mode = LDPM_LAUNCH_PAIRS;
    PersistCtl pctl;          // device words arrive / status of the persistent kernel's grid barriers
    int persist_grid = 0;     // its grid (co-resident blocks), 0 until the mode is first chosen
    BatchLaw batch_law{};     // mixed-mode batches of 2..kParamSpecimens specimens: law constants for the
                              // kernel parameters of the FP32 facet pass (n = 0 otherwise)
    size_t rsize() const { return prec == LDPM_MIXED ? sizeof(float) : sizeof(double); }
    size_t r4size() const { return 4 * rsize(); }
};

namespace {

void free_model(ldpm_ctx *h)
{
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    void *ptrs[] = {h->dm.pstate, h->dm.pdyn, h->dm.pconst, h->dm.pm32, h->dm.bc_vel, h->dm.bc_vm, h->dm.f_ext,
                    h->dm.tet,
                    h->dm.geo,
                    h->dm.hist, h->dm.fout, h->dm.tvc, h->dm.ent, h->dm.row, h->dm.stab, h->dm.tile_spec, h->dm.law, h->dm.spec,
                    h->dm.step, h->dm.flag, h->d_partial, h->d_out16, h->dm.pf, h->d_umap, h->d_scratch, h->d_ticket,
                    h->d_pmap, h->pctl.arrive, h->pctl.status};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->h_out16) cudaFreeHost(h->h_out16);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

template <class T>
int dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? LDPM_E_OOM : LDPM_E_CUDA, "cudaMalloc of %zu bytes: %s",
                    count * sizeof(T), cudaGetErrorString(e));
    }
    return LDPM_OK;
}

int check_material(const ldpm_material &m)
{
    const double v[] = {m.rho, m.E0, m.alpha, m.sigma_t, m.l_t, m.r_st, m.n_t, m.sigma_c0, m.Hc0_E0, m.Hc1_E0,
                        m.kc0, m.kc1, m.kc2, m.kc3, m.mu0, m.mu_inf, m.sigma_N0, m.Ed_E0, m.beta, m.k_t, m.r_s};
    for (double x : v)
        if (!std::isfinite(x)) return fail(LDPM_E_INVALID_ARG, "material parameter is not finite");
    if (!(m.rho > 0 && m.E0 > 0 && m.alpha > 0 && m.sigma_t > 0 && m.l_t > 0 && m.r_st > 0 && m.n_t >= 0 &&
          m.sigma_c0 > 0 && m.kc0 >= 1 && m.kc3 > 0 && m.sigma_N0 > 0 && m.Ed_E0 > 0 && m.k_t >= 0 && m.r_s >= 0))
        return fail(LDPM_E_INVALID_ARG, "material: rho, E0, alpha, sigma_t, l_t, r_st, sigma_c0, kc3, sigma_N0, "
                                        "Ed_E0 must be > 0; n_t, k_t, r_s >= 0; kc0 >= 1");
    if (m.reserved != 0) return fail(LDPM_E_INVALID_ARG, "material.reserved must be 0");
    return LDPM_OK;
}

// Per-specimen host preprocessing into the internal layout.  Writes this specimen's slices of the
// host mirrors of every device array.
struct HostArrays {
    std::vector<double> pstate, pdyn, pconst, bc_vel, bc_vm, f_ext;
    std::vector<int4> tet;
    std::unique_ptr<double[]> geo64;  // [Fint][4] before rounding to R (padding facets zeroed)
    std::vector<int32_t> row;
    std::vector<int64_t> ent_id;  // CSR payload: tetrahedron vertex slot 4 * tet + vertex
    std::vector<int32_t> tile_spec;
    bool any_fext = false;
};

int prepare_specimen(int s, const ldpm_geometry &g, const ldpm_options &o, SpecHost &S, HostArrays &H,
                     std::vector<double> &x_int, std::vector<double> &inv_mass, std::vector<double> &pconst_h)
{
    const int32_t N = g.n_particles, T = g.n_tets, F = g.n_facets;
    if (N < 4 || T < 1 || F != 12 * T)
        return fail(LDPM_E_BAD_GEOMETRY, "specimen %d: need N >= 4, T >= 1 and F == 12 T (N=%d T=%d F=%d)", s, N,
                    T, F);
    if (!g.x || !g.tet || !g.facet_pi || !g.facet_pj || !g.facet_tet || !g.facet_vtx)
        return fail(LDPM_E_INVALID_ARG, "specimen %d: geometry array is NULL", s);
    if (!g.diameter && !g.inertia)
        return fail(LDPM_E_INVALID_ARG, "specimen %d: need diameter or inertia", s);
    const ldpm_material &mat = S.mat;
    // ---- tetrahedra
    std::vector<double> tvol(T);
    auto tet_check = [&](int32_t t) -> int {  // 0 ok, 1 index out of range, 2 repeated, 3 volume
        const int32_t *v = g.tet + 4 * (size_t)t;
        for (int i = 0; i < 4; ++i) {
            if (v[i] < 0 || v[i] >= N) return 1;
            for (int k = 0; k < i; ++k)
                if (v[k] == v[i]) return 2;
        }
        double d[3][3];
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 3; ++a) d[i][a] = g.x[3 * (size_t)v[i + 1] + a] - g.x[3 * (size_t)v[0] + a];
        const double det = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                           d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                           d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
        if (!(std::fabs(det) > 0) || !std::isfinite(det)) return 3;
        tvol[t] = std::fabs(det) / 6.0;
        return 0;
    };
    const int64_t bad_t = parallel_min(T, [&](int64_t t0, int64_t t1) -> int64_t {
        for (int64_t t = t0; t < t1; ++t)
            if (tet_check((int32_t)t)) return t;
        return (int64_t)T;
    });
    if (bad_t < T) {
        const int32_t t = (int32_t)bad_t;
        const int kind = tet_check(t);
        if (kind == 1) return fail(LDPM_E_BAD_GEOMETRY, "tet %d: particle index out of range", t);
        if (kind == 2) return fail(LDPM_E_BAD_GEOMETRY, "tet %d: repeated particle", t);
        return fail(LDPM_E_BAD_GEOMETRY, "tet %d: zero or non-finite volume", t);
    }
    for (int32_t i = 0; i < 3 * N; ++i)
        if (!std::isfinite(g.x[i])) return fail(LDPM_E_BAD_GEOMETRY, "particle coordinate is not finite");
    // ---- Morton order of particles and tetrahedra
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, span[3];
    for (int32_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], g.x[3 * (size_t)i + a]);
            hi[a] = std::max(hi[a], g.x[3 * (size_t)i + a]);
        }
    for (int a = 0; a < 3; ++a) span[a] = hi[a] - lo[a];
    std::vector<uint32_t> key(N);
    for (int32_t i = 0; i < N; ++i) key[i] = morton3(g.x + 3 * (size_t)i, lo, span);
    S.perm_p = order_by_key(key);
    S.inv_p.assign(N, 0);
    for (int32_t r = 0; r < N; ++r) S.inv_p[S.perm_p[r]] = r;
    std::vector<uint32_t> tkey(T);
    parallel_min(T, [&](int64_t t0, int64_t t1) -> int64_t {
        for (int64_t t = t0; t < t1; ++t) {
            double c[3] = {0, 0, 0};
            for (int i = 0; i < 4; ++i)
                for (int a = 0; a < 3; ++a) c[a] += 0.25 * g.x[3 * (size_t)g.tet[4 * (size_t)t + i] + a];
            tkey[t] = morton3(c, lo, span);
        }
        return 0;
    });
    const std::vector<int32_t> perm_t = order_by_key(tkey);
    std::vector<int32_t> inv_t(T);
    for (int32_t r = 0; r < T; ++r) inv_t[perm_t[r]] = r;
    S.tmap.resize(T);
    for (int32_t t = 0; t < T; ++t) S.tmap[t] = S.t0 + inv_t[t];

    // ---- particles: positions, lumped mass (Sec. 3.2.5), BCs, initial velocity
    std::vector<double> mass(N, 0.0);
    for (int32_t t = 0; t < T; ++t)
        for (int i = 0; i < 4; ++i) mass[g.tet[4 * (size_t)t + i]] += mat.rho * tvol[t] / 4.0;
    double dpos = INFINITY;
    if (g.diameter)
        for (int32_t i = 0; i < N; ++i)
            if (g.diameter[i] > 0 && g.diameter[i] < dpos) dpos = g.diameter[i];
    S.W_kin0 = 0.0;
    for (int32_t i = 0; i < N; ++i) {
        const int32_t r = S.inv_p[i];
        const size_t P = (size_t)S.p0 + r;
        const double mi = g.mass ? g.mass[i] : mass[i];
        double md[6];
        for (int a = 0; a < 3; ++a) {
            md[a] = mi;
            if (g.inertia) {
                md[3 + a] = g.inertia[3 * (size_t)i + a];
            } else {
                const double d = g.diameter[i] > 0 ? g.diameter[i] : dpos;
                md[3 + a] = mi * d * d / 10.0;
            }
        }
        uint64_t bits = 0;
        for (int k = 0; k < 6; ++k) {
            if (!(md[k] > 0) || !std::isfinite(md[k]))
                return fail(LDPM_E_BAD_GEOMETRY, "particle %d: non-positive mass or inertia", i);
            const int mk = o.bc_mask ? o.bc_mask[6 * (size_t)i + k] : 0;
            if (mk < 0 || mk > 2) return fail(LDPM_E_INVALID_ARG, "bc_mask must be 0, 1 or 2");
            bits |= (uint64_t)mk << (8 * k);
            inv_mass[6 * P + k] = 1.0 / md[k];
            pconst_h[8 * P + k] = 1.0 / md[k];
            const double vb = o.bc_vel ? o.bc_vel[6 * (size_t)i + k] : 0.0;
            H.bc_vel[6 * P + k] = vb;
            H.bc_vm[6 * P + k] = vb * md[k];
            if (o.f_ext) {
                H.f_ext[6 * P + k] = o.f_ext[6 * (size_t)i + k];
                H.any_fext = true;
            }
            double v = o.v0 ? o.v0[6 * (size_t)i + k] : 0.0;
            if (mk == 1) v = 0.0;
            if (mk == 2) v = vb * (o.ramp_time <= 0 ? 1.0 : 0.0);
            H.pstate[16 * P + 9 + k] = v;
            S.W_kin0 += 0.5 * md[k] * v * v;
        }
        int64_t sb;
        std::memcpy(&pconst_h[8 * P + 6], &bits, 8);
        sb = s;
        std::memcpy(&pconst_h[8 * P + 7], &sb, 8);
        for (int a = 0; a < 3; ++a) {
            H.pstate[16 * P + a] = g.x[3 * (size_t)i + a];
            x_int[3 * P + a] = g.x[3 * (size_t)i + a];
        }
    }
    // ---- tetrahedra in Morton order (padding tetrahedra keep particle id -1)
    for (int32_t r = 0; r < T; ++r) {
        const int32_t *v = g.tet + 4 * (size_t)perm_t[r];
        H.tet[(size_t)S.t0 + r] = make_int4(S.p0 + S.inv_p[v[0]], S.p0 + S.inv_p[v[1]], S.p0 + S.inv_p[v[2]],
                                            S.p0 + S.inv_p[v[3]]);
    }
    for (int32_t r = 0; r < S.T_pad / kTile; ++r) H.tile_spec[S.t0 / kTile + r] = s;
    // ---- facets: slot = 2 * edge + k within the tetrahedron; the first of an edge's two facets in the
    // caller's order takes the lower slot.  Three passes on host threads: the facet's tetrahedron and
    // edge; the slots (each thread owns a range of tetrahedra and scans the facets in the caller's
    // order); the geometry.  Each check reports the first failing facet in the caller's order, as one
    // sequential loop would.
    S.fmap.assign(F, -1);
    S.fswap.assign(F, 0);
    std::vector<int32_t> rank(F);  // Morton rank of the facet's tetrahedron
    std::vector<uint8_t> lalb(F);  // local vertex indices la | lb << 2, edge << 4
    // the slot pass below runs parallel_min over the T ranks: owner[k] is the thread whose range
    // holds the facet's rank, so each thread scans one byte per facet
    const int64_t rank_chunk = ((int64_t)T + host_threads(T) - 1) / host_threads(T);
    std::vector<uint8_t> owner(F);
    int kind1 = 0;
    const int64_t bad1 = parallel_min(F, [&](int64_t lo, int64_t hi) -> int64_t {
        for (int64_t k = lo; k < hi; ++k) {
            const int32_t t = g.facet_tet[k];
            if (t < 0 || t >= T) return k;
            const int32_t *v = g.tet + 4 * (size_t)t;
            int la = -1, lb = -1;
            for (int i = 0; i < 4; ++i) {
                if (v[i] == g.facet_pi[k]) la = i;
                if (v[i] == g.facet_pj[k]) lb = i;
            }
            if (la < 0 || lb < 0 || la == lb) return k;
            rank[k] = inv_t[t];
            owner[k] = (uint8_t)(inv_t[t] / rank_chunk);
            lalb[k] = (uint8_t)(la | (lb << 2) | (edge_of(la, lb) << 4));
        }
        return (int64_t)F;
    });
    if (bad1 < F) {
        const int32_t t = g.facet_tet[bad1];
        kind1 = (t < 0 || t >= T) ? 1 : 2;
    }
    // Facets compete for slots only within their tetrahedron: each thread owns a range of Morton
    // ranks and scans all facets in the caller's order, taking those of its tetrahedra.
    std::vector<uint8_t> used((size_t)T * 12, 0);
    const int64_t bad2 = parallel_min(T, [&](int64_t r0, int64_t r1) -> int64_t {
        const uint8_t me = (uint8_t)(r0 / rank_chunk);
        const bool one_chunk = r1 - r0 <= rank_chunk;  // false only when run on a single thread
        int64_t first = bad1;
        for (int64_t k = 0; k < bad1; ++k) {
            if (one_chunk ? owner[k] != me : (rank[k] < r0 || rank[k] >= r1)) continue;
            const int64_t rt = rank[k];
            int slot = 2 * (lalb[k] >> 4);
            if (used[(size_t)rt * 12 + slot]) ++slot;
            if (used[(size_t)rt * 12 + slot]) {
                first = k;
                break;
            }
            used[(size_t)rt * 12 + slot] = 1;
            S.fmap[k] = ((int64_t)S.t0 + rt) * 12 + slot;
            S.fswap[k] = (lalb[k] & 3) > ((lalb[k] >> 2) & 3);
        }
        return first;
    });
    const int64_t upto = std::min(bad1, bad2);
    const int64_t bad3 = parallel_min(upto, [&](int64_t lo, int64_t hi) -> int64_t {
        for (int64_t k = lo; k < hi; ++k) {
            const int32_t *v = g.tet + 4 * (size_t)g.facet_tet[k];
            const int la = lalb[k] & 3, lb = (lalb[k] >> 2) & 3;
            const int64_t fi = S.fmap[k];
            // geometry from the internal first vertex a = min(la, lb)
            const int32_t pa = v[std::min(la, lb)], pb = v[std::max(la, lb)];
            const double *xa = g.x + 3 * (size_t)pa, *xb = g.x + 3 * (size_t)pb;
            const double *p0 = g.facet_vtx + 9 * (size_t)k;
            double dd[3], e1[3], e2[3], xc[3];
            for (int a = 0; a < 3; ++a) {
                dd[a] = xb[a] - xa[a];
                e1[a] = p0[3 + a] - p0[a];
                e2[a] = p0[6 + a] - p0[a];
                xc[a] = (p0[a] + p0[3 + a] + p0[6 + a]) / 3.0;
            }
            const double l = std::sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
            const double nc[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                  e1[0] * e2[1] - e1[1] * e2[0]};
            const double twoA0 = std::sqrt(nc[0] * nc[0] + nc[1] * nc[1] + nc[2] * nc[2]);
            if (!(l > 0) || !(twoA0 > 0) || !std::isfinite(twoA0)) return k;
            if (!(l < mat.l_t)) return k;
            // projected area A = A0 |n . n0| (Sec. 2)
            const double A = 0.5 * std::fabs((dd[0] * nc[0] + dd[1] * nc[1] + dd[2] * nc[2]) / l);
            for (int a = 0; a < 3; ++a) H.geo64[4 * (size_t)fi + a] = xc[a] - xa[a];
            H.geo64[4 * (size_t)fi + 3] = A;
        }
        return upto;
    });
    if (bad3 < upto) {  // the same two checks again, for the message
        const int64_t k = bad3;
        const int32_t *v = g.tet + 4 * (size_t)g.facet_tet[k];
        const int la = lalb[k] & 3, lb = (lalb[k] >> 2) & 3;
        const double *xa = g.x + 3 * (size_t)v[std::min(la, lb)], *xb = g.x + 3 * (size_t)v[std::max(la, lb)];
        const double *p0 = g.facet_vtx + 9 * (size_t)k;
        double l2 = 0.0, e1[3], e2[3];
        for (int a = 0; a < 3; ++a) {
            l2 += (xb[a] - xa[a]) * (xb[a] - xa[a]);
            e1[a] = p0[3 + a] - p0[a];
            e2[a] = p0[6 + a] - p0[a];
        }
        const double l = std::sqrt(l2);
        const double nc[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                              e1[0] * e2[1] - e1[1] * e2[0]};
        const double twoA0 = std::sqrt(nc[0] * nc[0] + nc[1] * nc[1] + nc[2] * nc[2]);
        if (!(l > 0) || !(twoA0 > 0) || !std::isfinite(twoA0))
            return fail(LDPM_E_BAD_GEOMETRY, "facet %lld: zero edge length or facet area", (long long)k);
        return fail(LDPM_E_BAD_GEOMETRY, "facet %lld: edge length %g >= l_t (softening modulus undefined)",
                    (long long)k, l);
    }
    if (bad2 < bad1)
        return fail(LDPM_E_BAD_GEOMETRY, "tetrahedron %d: more than 2 facets on one edge", g.facet_tet[bad2]);
    if (kind1 == 1) return fail(LDPM_E_BAD_GEOMETRY, "facet %lld: tetrahedron index out of range", (long long)bad1);
    if (kind1 == 2)
        return fail(LDPM_E_BAD_GEOMETRY, "facet %lld: I and J must be two vertices of its tetrahedron", (long long)bad1);
    const int64_t bad_r = parallel_min(T, [&](int64_t r0, int64_t r1) -> int64_t {
        for (int64_t r = r0; r < r1; ++r)
            for (int sl = 0; sl < 12; ++sl)
                if (!used[(size_t)r * 12 + sl]) return r;
        return (int64_t)T;
    });
    if (bad_r < T)
        return fail(LDPM_E_BAD_GEOMETRY, "tetrahedron %d: edge without its two facets", perm_t[bad_r]);
    return LDPM_OK;
}

template <class R>
int upload_facets(ldpm_ctx *h, const HostArrays &H, int64_t Fint)
{
    using T4 = R4<R>;
    std::vector<T4> geo(Fint);
    parallel_min(Fint, [&](int64_t f0, int64_t f1) -> int64_t {
        for (int64_t f = f0; f < f1; ++f) {
            geo[f].x = R(H.geo64[4 * f]);
            geo[f].y = R(H.geo64[4 * f + 1]);
            geo[f].z = R(H.geo64[4 * f + 2]);
            geo[f].w = R(H.geo64[4 * f + 3]);
        }
        return 0;
    });
    const int64_t nent = H.ent_id.size();
    std::vector<int32_t> ent(nent);
    for (int64_t r = 0; r < nent; ++r) ent[r] = (int32_t)H.ent_id[r];
    int rc;
    const int64_t T = Fint / 12;
    if ((rc = dalloc((T4 **)&h->dm.geo, Fint)) || (rc = dalloc((T4 **)&h->dm.hist, Fint)) ||
        (rc = dalloc((T4 **)&h->dm.fout, Fint)) || (rc = dalloc((R **)&h->dm.tvc, 24 * T)) ||
        (rc = dalloc((int32_t **)&h->dm.ent, std::max<int64_t>(nent, 1))))
        return rc;
    CU(cudaMemcpy(h->dm.geo, geo.data(), Fint * sizeof(T4), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->dm.ent, ent.data(), nent * sizeof(int32_t), cudaMemcpyHostToDevice));
    CU(cudaMemset(h->dm.tvc, 0, 24 * T * sizeof(R)));
    CU(cudaMemset(h->dm.hist, 0, Fint * sizeof(T4)));
    CU(cudaMemset(h->dm.fout, 0, Fint * sizeof(T4)));
    std::vector<LawConst<R>> law(h->sp.size());
    for (size_t s = 0; s < h->sp.size(); ++s) law_const<R>(h->sp[s].mat, h->sp[s].dt, law[s]);
    if ((rc = dalloc((LawConst<R> **)&h->dm.law, law.size()))) return rc;
    CU(cudaMemcpy(h->dm.law, law.data(), law.size() * sizeof(LawConst<R>), cudaMemcpyHostToDevice));
    return LDPM_OK;
}

int update_law(ldpm_ctx *h)
{
    if (h->prec == LDPM_MIXED) {
        std::vector<LawConst<float>> law(h->sp.size());
        for (size_t s = 0; s < h->sp.size(); ++s) law_const<float>(h->sp[s].mat, h->sp[s].dt, law[s]);
        CU(cudaMemcpy(h->dm.law, law.data(), law.size() * sizeof(law[0]), cudaMemcpyHostToDevice));
        BatchLaw bl{};
        const int n = (int)h->sp.size();
        if (n > 1 && n <= kParamSpecimens) {
            bl.n = n;
            for (int s = 0; s < n; ++s) {
                bl.t0[s] = h->sp[s].t0;
                bl.law[s] = law[s];
            }
            bl.t0[n] = h->dm.T;
        }
        if (std::memcmp(&h->dm.law1, &law[0], sizeof(law[0])) != 0 || std::memcmp(&h->batch_law, &bl, sizeof(bl)) != 0) {
            // the copies travel in the kernel parameters: captured launches hold the old ones
            CU(cudaStreamSynchronize(h->stream));
            for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
            h->graphs.clear();
            h->dm.law1 = law[0];
            h->batch_law = bl;
        }
    } else {
        std::vector<LawConst<double>> law(h->sp.size());
        for (size_t s = 0; s < h->sp.size(); ++s) law_const<double>(h->sp[s].mat, h->sp[s].dt, law[s]);
        CU(cudaMemcpy(h->dm.law, law.data(), law.size() * sizeof(law[0]), cudaMemcpyHostToDevice));
    }
    std::vector<SpecDyn> sd(h->sp.size());
    for (size_t s = 0; s < h->sp.size(); ++s) {
        const double T = h->sp[s].ramp_time, dt = h->sp[s].dt;
        sd[s] = SpecDyn{dt, T, 1.0 / dt, T > 0 ? 1.0 / T : 0.0, 0.5 * dt};
    }
    CU(cudaMemcpy(h->dm.spec, sd.data(), sd.size() * sizeof(SpecDyn), cudaMemcpyHostToDevice));
    return LDPM_OK;
}

int launch_facet_any(ldpm_ctx *h, int mode, const void *pst)
{
    cudaError_t e = h->prec == LDPM_MIXED
                        ? launch_facet<float>(h->dm, mode, pst, h->stream, h->batch_law.n ? &h->batch_law : nullptr)
                        : launch_facet<double>(h->dm, mode, pst, h->stream);
    if (e != cudaSuccess) return fail(LDPM_E_CUDA, "facet pass launch: %s", cudaGetErrorString(e));
    return LDPM_OK;
}

int launch_gather_any(ldpm_ctx *h, int mode, double *out6)
{
    cudaError_t e = h->prec == LDPM_MIXED ? launch_gather<float>(h->dm, mode, out6, h->stream)
                                          : launch_gather<double>(h->dm, mode, out6, h->stream);
    if (e != cudaSuccess) return fail(LDPM_E_CUDA, "particle pass launch: %s", cudaGetErrorString(e));
    return LDPM_OK;
}

// Rebuild the node force sums of the current state from the stored tractions (f = sum A P t).
int forces_from_history(ldpm_ctx *h)
{
    int rc;
    double *out6 = nullptr;
    if ((rc = dalloc(&out6, 6 * (size_t)h->dm.N))) return rc;
    if ((rc = launch_facet_any(h, FACET_FROM_HIST, nullptr)) || (rc = launch_gather_any(h, GATHER_ASSEMBLE, out6))) {
        cudaFree(out6);
        return rc;
    }
    cudaError_t e = cudaMemcpy2DAsync(h->dm.pdyn, 8 * sizeof(double), out6, 6 * sizeof(double), 6 * sizeof(double),
                                      h->dm.N, cudaMemcpyDeviceToDevice, h->stream);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    cudaFree(out6);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(LDPM_E_CUDA, "force rebuild: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return LDPM_OK;
}

// Largest eigenvalue of M^-1 K per specimen by power iteration; the elastic operator is one facet
// pass (t = E e at displacement x) plus one assembly.  Host-side vector algebra, device mat-vec.
int estimate_dt(ldpm_ctx *h, std::vector<double> &lam)
{
    const int32_t N = h->dm.N;
    const size_t n6 = 6 * (size_t)N;
    int rc;
    const bool mixed = h->prec == LDPM_MIXED;
    const size_t rec = mixed ? (size_t)kMirror * sizeof(float) : 16 * sizeof(double);
    void *pst = nullptr;
    double *out6 = nullptr;
    if ((rc = dalloc((char **)&pst, rec * (size_t)N)) || (rc = dalloc(&out6, n6))) {
        cudaFree(pst);
        return rc;
    }
    // displacement x (iteration vector) on the reference positions; zero velocity
    std::vector<double> ps(16 * (size_t)N, 0.0), x(n6), f(n6);
    std::vector<float> pm(mixed ? (size_t)kMirror * N : 0, 0.0f);
    for (int32_t p = 0; p < N; ++p)
        for (int a = 0; a < 3; ++a) {
            const double xv = h->x_int[3 * (size_t)p + a];
            ps[16 * (size_t)p + a] = xv;
            if (mixed) {
                const float hi = (float)xv;
                pm[kMirror * (size_t)p + a] = hi;
                pm[kMirror * (size_t)p + 3 + a] = (float)(xv - (double)hi);
            }
        }
    std::mt19937_64 rng(12345);
    std::normal_distribution<double> nd;
    for (auto &v : x) v = nd(rng);
    const int nsp = (int)h->sp.size();
    lam.assign(nsp, 0.0);
    std::vector<double> prev(nsp, 0.0);
    const int max_it = 400;
    for (int it = 0; it < max_it; ++it) {
        for (int s = 0; s < nsp; ++s) {
            const size_t a = 6 * (size_t)h->sp[s].p0, b = a + 6 * (size_t)h->sp[s].N;
            double nrm = 0;
            for (size_t i = a; i < b; ++i) nrm += x[i] * x[i] / h->inv_mass[i];
            nrm = std::sqrt(nrm);
            for (size_t i = a; i < b; ++i) x[i] /= nrm;
        }
        for (int32_t p = 0; p < N; ++p)
            for (int k = 0; k < 6; ++k) {
                const double u = x[6 * (size_t)p + k];
                ps[16 * (size_t)p + 3 + k] = u;
                if (mixed) {
                    float *r = &pm[kMirror * (size_t)p];
                    if (k < 3) {
                        const float hi = (float)u;
                        r[6 + k] = hi;
                        r[9 + k] = (float)(u - (double)hi);
                    } else {
                        r[12 + k - 3] = (float)u;
                    }
                }
            }
        if (mixed)
            CU(cudaMemcpyAsync(pst, pm.data(), pm.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        else
            CU(cudaMemcpyAsync(pst, ps.data(), ps.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        if ((rc = launch_facet_any(h, FACET_ELASTIC, pst)) || (rc = launch_gather_any(h, GATHER_ASSEMBLE, out6))) break;
        CU(cudaMemcpyAsync(f.data(), out6, n6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        bool done = it >= 30;
        for (int s = 0; s < nsp; ++s) {
            const size_t a = 6 * (size_t)h->sp[s].p0, b = a + 6 * (size_t)h->sp[s].N;
            double xkx = 0;
            for (size_t i = a; i < b; ++i) xkx -= x[i] * f[i];
            lam[s] = xkx;  // x^T M x = 1
            if (std::fabs(lam[s] - prev[s]) > 1e-5 * std::fabs(lam[s])) done = false;
            prev[s] = lam[s];
        }
        for (size_t i = 0; i < n6; ++i) x[i] = -f[i] * h->inv_mass[i];
        if (done) break;
    }
    cudaFree(pst);
    cudaFree(out6);
    if (rc) return rc;
    for (int s = 0; s < nsp; ++s)
        if (!(lam[s] > 0) || !std::isfinite(lam[s]))
            return fail(LDPM_E_BAD_GEOMETRY, "specimen %d: critical step estimate failed (lambda %g)", s, lam[s]);
    return LDPM_OK;
}

int kick(ldpm_ctx *h);
int enqueue_direct(ldpm_ctx *h, int64_t nsteps);
int enqueue_steps(ldpm_ctx *h, int64_t nsteps);
int set_launch_mode(ldpm_ctx *h, int mode);

// Launch-shape autotuner: times each candidate (tetrahedra per facet-pass block x lanes per particle)
// on the model itself for a few steps, restoring the complete mutable state after every trial, and
// keeps the fastest; then times that shape's graph-replayed launch pairs against the persistent launch
// the same way and keeps the faster mode.  Results stay deterministic for the chosen shape: the facet-pass shape does not
// change any arithmetic, the lanes per particle change the order of a particle's sums (rounding-level
// differences between shapes).
int autotune(ldpm_ctx *h)
{
    DeviceModel &dm = h->dm;
    const size_t n_ps = 16 * (size_t)dm.N * 8, n_pd = 8 * (size_t)dm.N * 8, n_pm = dm.pm32 ? (size_t)kMirror * dm.N * 4 : 0;
    const size_t n_h = 12 * (size_t)dm.T * h->r4size();
    char *bk = nullptr;
    int rc;
    if ((rc = dalloc(&bk, n_ps + n_pd + n_pm + n_h + 16))) return rc;
    auto save = [&](bool to_backup) -> cudaError_t {
        char *b = bk;
        void *dst[5] = {b, b + n_ps, b + n_ps + n_pd, b + n_ps + n_pd + n_pm, b + n_ps + n_pd + n_pm + n_h};
        void *src[5] = {dm.pstate, dm.pdyn, dm.pm32, dm.hist, dm.step};
        const size_t sz[5] = {n_ps, n_pd, n_pm, n_h, 8};
        for (int k = 0; k < 5; ++k) {
            if (!sz[k] || !src[k]) continue;
            cudaError_t e = to_backup ? cudaMemcpyAsync(dst[k], src[k], sz[k], cudaMemcpyDeviceToDevice, h->stream)
                                      : cudaMemcpyAsync(src[k], dst[k], sz[k], cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int tets[3] = {8, 16, 32}, lanes[2] = {8, 16};
    float best = 1e30f;
    int bt = dm.tets_per_block, bl = dm.gather_lanes;
    cudaError_t e = save(true);
    for (int ti = 0; ti < 3 && e == cudaSuccess && rc == 0; ++ti)
        for (int li = 0; li < 2 && e == cudaSuccess && rc == 0; ++li) {
            dm.tets_per_block = tets[ti];
            dm.gather_lanes = lanes[li];
            if ((rc = enqueue_direct(h, 1))) break;  // warm-up
            e = cudaEventRecord(a, h->stream);
            if (e == cudaSuccess && !(rc = enqueue_direct(h, 3))) e = cudaEventRecord(b, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                bt = tets[ti];
                bl = lanes[li];
            }
            if (e == cudaSuccess) e = save(false);
        }
    dm.tets_per_block = bt;
    dm.gather_lanes = bl;
    // launch mode: the chosen launch pairs replayed from CUDA graphs against the persistent launch, each
    // timed over the same steps from the same state (a warm-up call first captures the graphs)
    float t_mode[3] = {0.f, 0.f, 0.f};
    for (int mode = LDPM_LAUNCH_PAIRS; mode <= LDPM_LAUNCH_PERSISTENT && e == cudaSuccess && rc == 0; ++mode) {
        if (set_launch_mode(h, mode) != LDPM_OK) {  // no co-resident persistent grid: pairs only
            set_last_error("");
            t_mode[mode] = 1e30f;
            continue;
        }
        for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
        h->graphs.clear();
        constexpr int kTrial = 8;
        if ((rc = enqueue_steps(h, kTrial))) break;
        e = cudaEventRecord(a, h->stream);
        if (e == cudaSuccess && !(rc = enqueue_steps(h, kTrial))) e = cudaEventRecord(b, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_mode[mode], a, b);
        if (e == cudaSuccess) e = save(false);
    }
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    if (rc == 0 && e == cudaSuccess)
        rc = set_launch_mode(h, t_mode[LDPM_LAUNCH_PERSISTENT] < t_mode[LDPM_LAUNCH_PAIRS] ? LDPM_LAUNCH_PERSISTENT
                                                                                         : LDPM_LAUNCH_PAIRS);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(bk);
    if (rc) return rc;
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(LDPM_E_CUDA, "autotune: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return LDPM_OK;
}

int create_model(int n, const ldpm_geometry *geoms, const ldpm_material *mats, const ldpm_options *opts,
                 ldpm_t *out)
{
    if (!out) return fail(LDPM_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !geoms || !mats || !opts) return fail(LDPM_E_INVALID_ARG, "need n >= 1 and non-NULL arrays");
    const ldpm_options &o0 = opts[0];
    if (o0.precision != LDPM_FP64 && o0.precision != LDPM_MIXED)
        return fail(LDPM_E_INVALID_ARG, "precision must be LDPM_FP64 or LDPM_MIXED");
    for (int s = 0; s < n; ++s) {
        if (opts[s].precision != o0.precision) return fail(LDPM_E_INVALID_ARG, "specimens must share the precision");
        if (opts[s].autotune != 0 && opts[s].autotune != 1) return fail(LDPM_E_INVALID_ARG, "options.autotune must be 0 or 1");
        if (!std::isfinite(opts[s].dt) || !std::isfinite(opts[s].ramp_time))
            return fail(LDPM_E_INVALID_ARG, "dt and ramp_time must be finite");
        int rc = check_material(mats[s]);
        if (rc) return rc;
    }
    std::unique_ptr<ldpm_ctx> h(new (std::nothrow) ldpm_ctx);
    if (!h) return fail(LDPM_E_OOM, "host allocation");
    h->prec = o0.precision;
    h->graph_chunk = o0.graph_chunk == 0 ? 32 : o0.graph_chunk;
    h->sp.resize(n);
    int64_t Np = 0, Tp = 0;
    for (int s = 0; s < n; ++s) {
        SpecHost &S = h->sp[s];
        S.N = geoms[s].n_particles;
        S.T = geoms[s].n_tets;
        S.F = geoms[s].n_facets;
        if (S.N < 4 || S.T < 1 || (int64_t)S.F != 12 * (int64_t)S.T)
            return fail(LDPM_E_BAD_GEOMETRY, "specimen %d: need N >= 4, T >= 1 and F == 12 T", s);
        S.mat = mats[s];
        S.ramp_time = opts[s].ramp_time;
        S.dt = opts[s].dt;
        S.p0 = (int32_t)Np;
        S.t0 = (int32_t)Tp;
        S.T_pad = (S.T + kTile - 1) / kTile * kTile;
        Np += S.N;
        Tp += S.T_pad;
    }
    if (Np > INT32_MAX / 2 || 24 * Tp > (int64_t)INT32_MAX)
        return fail(LDPM_E_INVALID_ARG, "specimen too large for 32-bit slot ids");
    const int32_t N = (int32_t)Np, T = (int32_t)Tp;
    const int64_t Fint = 12 * (int64_t)T;
    HostArrays H;
    H.pstate.assign(16 * (size_t)N, 0.0);
    H.pdyn.assign(8 * (size_t)N, 0.0);
    H.bc_vel.assign(6 * (size_t)N, 0.0);
    H.bc_vm.assign(6 * (size_t)N, 0.0);
    H.f_ext.assign(6 * (size_t)N, 0.0);
    H.tet.assign(T, make_int4(-1, -1, -1, -1));
    H.geo64.reset(new double[4 * (size_t)Fint]);  // every facet of a real tetrahedron is written
    H.tile_spec.assign(T / kTile, 0);
    h->x_int.assign(3 * (size_t)N, 0.0);
    h->inv_mass.assign(6 * (size_t)N, 0.0);
    h->pconst_h.assign(8 * (size_t)N, 0.0);
    for (int s = 0; s < n; ++s) {
        int rc = prepare_specimen(s, geoms[s], opts[s], h->sp[s], H, h->x_int, h->inv_mass, h->pconst_h);
        if (rc) return rc;
        const SpecHost &S = h->sp[s];
        std::fill(H.geo64.get() + 48 * ((size_t)S.t0 + S.T), H.geo64.get() + 48 * ((size_t)S.t0 + S.T_pad), 0.0);
    }
    // ---- CSR of facet ends, ascending facet id within each particle (fixed summation order)
    H.row.assign((size_t)N + 1, 0);
    for (int64_t t = 0; t < T; ++t) {
        const int4 v = H.tet[t];
        if (v.x < 0) continue;
        H.row[v.x + 1]++;
        H.row[v.y + 1]++;
        H.row[v.z + 1]++;
        H.row[v.w + 1]++;
    }
    for (int32_t p = 0; p < N; ++p) H.row[p + 1] += H.row[p];
    H.ent_id.assign(H.row[N], 0);
    {
        // ascending tetrahedron within each particle: the fixed summation order
        std::vector<int32_t> pos(H.row.begin(), H.row.end() - 1);
        for (int64_t t = 0; t < T; ++t) {
            const int4 v = H.tet[t];
            if (v.x < 0) continue;
            const int vv[4] = {v.x, v.y, v.z, v.w};
            for (int k = 0; k < 4; ++k) H.ent_id[pos[vv[k]]++] = 4 * t + k;
        }
    }
    // ---- caller's facet order -> internal facet (with the orientation flip in bit 0)
    std::vector<int32_t> umap;
    h->ufoff.assign(n + 1, 0);
    for (int s = 0; s < n; ++s) h->ufoff[s + 1] = h->ufoff[s] + h->sp[s].F;
    umap.resize((size_t)h->ufoff[n]);
    for (int s = 0; s < n; ++s) {
        const SpecHost &S = h->sp[s];
        int32_t *dst = umap.data() + h->ufoff[s];
        parallel_min(S.F, [&](int64_t k0, int64_t k1) -> int64_t {
            for (int64_t k = k0; k < k1; ++k) dst[k] = (int32_t)(2 * S.fmap[k] + S.fswap[k]);
            return 0;
        });
    }
    // ---- device
    int dev = o0.device;
    if (dev < 0) CU(cudaGetDevice(&dev));
    CU(cudaSetDevice(dev));
    h->device = dev;
    if (o0.cuda_stream) {
        h->stream = (cudaStream_t)o0.cuda_stream;
    } else {
        CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    ldpm_ctx *raw = h.get();
    struct Guard {
        ldpm_ctx *p;
        bool armed = true;
        ~Guard()
        {
            if (armed) free_model(p);
        }
    } guard{raw};
    DeviceModel &dm = h->dm;
    dm.N = N;
    dm.T = T;
    dm.n_spec = n;
    dm.tets_per_block = 8;  // measured fastest of 8/16/32 on GB300 (uniaxial_tension, mixed)
    dm.gather_lanes = 8;    // measured fastest of 8/16/32
    // Launch-shape overrides for tuning: LDPM_GATHER_LANES (8, 16, 32), LDPM_TETS_PER_BLOCK (8, 16, 32).
    if (const char *ev = std::getenv("LDPM_GATHER_LANES")) {
        const int v = std::atoi(ev);
        if (v == 8 || v == 16 || v == 32) dm.gather_lanes = v;
    }
    if (const char *ev = std::getenv("LDPM_TETS_PER_BLOCK")) {
        const int v = std::atoi(ev);
        if (v == 8 || v == 16 || v == 32) dm.tets_per_block = v;
    }
    if (const char *ev = std::getenv("LDPM_BLOCKS_PER_SM")) dm.blocks_per_sm = std::max(0, std::atoi(ev));
    int rc;
    if ((rc = dalloc(&dm.pstate, 16 * (size_t)N)) || (rc = dalloc(&dm.pdyn, 8 * (size_t)N)) ||
        (rc = dalloc(&dm.pconst, 8 * (size_t)N)) || (rc = dalloc(&dm.bc_vel, 6 * (size_t)N)) ||
        (rc = dalloc(&dm.bc_vm, 6 * (size_t)N)) ||
        (rc = dalloc(&dm.tet, (size_t)T)) || (rc = dalloc(&dm.row, (size_t)N + 1)) ||
        (rc = dalloc(&dm.stab, (size_t)kSlotTab * N)) ||
        (rc = dalloc(&dm.tile_spec, (size_t)T / kTile)) || (rc = dalloc(&dm.spec, (size_t)n)) ||
        (rc = dalloc(&dm.step, 1)) || (rc = dalloc(&dm.flag, 1)) || (rc = dalloc(&h->d_out16, 16)) ||
        (rc = dalloc(&h->d_partial, 16 * (size_t)((N + 255) / 256 + 1))) || (rc = dalloc(&h->d_umap, umap.size())) ||
        (rc = dalloc(&h->d_ticket, 1)) || (rc = dalloc(&h->d_pmap, (size_t)N)) ||
        (rc = dalloc(&h->pctl.arrive, 1)) || (rc = dalloc(&h->pctl.status, 1)))
        return rc;
    CU(cudaMemset(h->pctl.arrive, 0, sizeof(unsigned)));
    CU(cudaMemset(h->pctl.status, 0, sizeof(int32_t)));
    {
        std::vector<int32_t> pmap((size_t)N);
        size_t base = 0;
        for (const SpecHost &S : h->sp) {
            for (int32_t i = 0; i < S.N; ++i) pmap[base + i] = S.p0 + S.inv_p[i];
            base += S.N;
        }
        CU(cudaMemcpy(h->d_pmap, pmap.data(), pmap.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    CU(cudaMemset(h->d_ticket, 0, sizeof(unsigned)));
    CU(cudaMemcpy(h->d_umap, umap.data(), umap.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (H.any_fext) {
        if ((rc = dalloc(&dm.f_ext, 6 * (size_t)N))) return rc;
        CU(cudaMemcpy(dm.f_ext, H.f_ext.data(), H.f_ext.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (h->prec == LDPM_MIXED && (rc = dalloc(&dm.pm32, (size_t)kMirror * N))) return rc;
    CU(cudaMallocHost((void **)&h->h_out16, 16 * sizeof(double)));
    CU(cudaMemcpy(dm.pstate, H.pstate.data(), H.pstate.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dm.pdyn, H.pdyn.data(), H.pdyn.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dm.pconst, h->pconst_h.data(), h->pconst_h.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dm.bc_vel, H.bc_vel.data(), H.bc_vel.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dm.bc_vm, H.bc_vm.data(), H.bc_vm.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dm.tet, H.tet.data(), H.tet.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dm.row, H.row.data(), H.row.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    {
        // slot table: the first kSlotTab CSR entries of each particle, -1 after the row's end
        std::vector<int32_t> stab((size_t)kSlotTab * N, -1);
        parallel_min(N, [&](int64_t p0, int64_t p1) -> int64_t {
            for (int64_t p = p0; p < p1; ++p) {
                const int64_t r0 = H.row[p], n = std::min<int64_t>(H.row[p + 1] - r0, kSlotTab);
                for (int64_t j = 0; j < n; ++j) stab[(size_t)p * kSlotTab + j] = (int32_t)H.ent_id[r0 + j];
            }
            return 0;
        });
        CU(cudaMemcpy(dm.stab, stab.data(), stab.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    CU(cudaMemcpy(dm.tile_spec, H.tile_spec.data(), H.tile_spec.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CU(cudaMemset(dm.step, 0, sizeof(int64_t)));
    CU(cudaMemset(dm.flag, 0, sizeof(int32_t)));
    CU(launch_mirror(dm, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    for (auto &S : h->sp)
        if (!(S.dt > 0)) S.dt = 1.0;  // placeholder until estimated
    if (h->prec == LDPM_MIXED)
        rc = upload_facets<float>(raw, H, Fint);
    else
        rc = upload_facets<double>(raw, H, Fint);
    if (rc) return rc;
    if ((rc = update_law(raw))) return rc;
    // ---- time step: given, or dt_factor * 2 / sqrt(lambda_max)
    bool need = false;
    for (int s = 0; s < n; ++s) need |= !(opts[s].dt > 0);
    if (need) {
        std::vector<double> lam;
        if ((rc = estimate_dt(raw, lam))) return rc;
        for (int s = 0; s < n; ++s)
            if (!(opts[s].dt > 0)) {
                const double fac = opts[s].dt_factor > 0 ? opts[s].dt_factor : 0.9;
                h->sp[s].dt = fac * 2.0 / std::sqrt(lam[s]);
            }
        if ((rc = update_law(raw))) return rc;
        CU(cudaMemset(dm.fout, 0, Fint * h->r4size()));
    }
    // the library keeps the drifted state between calls: first half kick and drift of step 0
    if ((rc = kick(raw))) return rc;
    if (o0.autotune && (rc = autotune(raw))) return rc;
    CU(cudaDeviceSynchronize());
    guard.armed = false;
    *out = h.release();
    return LDPM_OK;
}

// nsteps explicit steps on the drifted state: facet pass, then the fused particle pass.
int enqueue_direct(ldpm_ctx *h, int64_t nsteps)
{
    int rc;
    for (int64_t i = 0; i < nsteps; ++i) {
        if ((rc = launch_facet_any(h, FACET_STEP, nullptr))) return rc;
        if ((rc = launch_gather_any(h, GATHER_STEP_MID, nullptr))) return rc;
    }
    return LDPM_OK;
}

int kick(ldpm_ctx *h)
{
    cudaError_t e = launch_kick(h->dm, h->stream);
    if (e != cudaSuccess) return fail(LDPM_E_CUDA, "kick launch: %s", cudaGetErrorString(e));
    return LDPM_OK;
}

int graph_for(ldpm_ctx *h, int64_t len, cudaGraphExec_t *exec)
{
    auto it = h->graphs.find(len);
    if (it != h->graphs.end()) {
        *exec = it->second;
        return LDPM_OK;
    }
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_direct(h, len);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(LDPM_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LDPM_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    h->graphs[len] = ex;
    *exec = ex;
    return LDPM_OK;
}

int enqueue_profiled(ldpm_ctx *h, int64_t nsteps)
{
    // three events per step (before the facet pass, between the passes, after the particle pass): the
    // two kernel times add up to the step's time, with no event between consecutive steps
    int rc;
    for (int64_t i = 0; i < nsteps; ++i) {
        cudaEvent_t ev[3];
        for (auto &e : ev) {
            if (cudaEventCreate(&e) != cudaSuccess) return fail(LDPM_E_CUDA, "event create failed");
            h->ev_pool.push_back(e);
        }
        const int i0 = (int)h->ev_pool.size() - 3;
        h->ev_pairs.push_back({1, i0, i0 + 1});
        h->ev_pairs.push_back({2, i0 + 1, i0 + 2});
        CU(cudaEventRecord(ev[0], h->stream));
        if ((rc = launch_facet_any(h, FACET_STEP, nullptr))) return rc;
        CU(cudaEventRecord(ev[1], h->stream));
        if ((rc = launch_gather_any(h, GATHER_STEP_MID, nullptr))) return rc;
        CU(cudaEventRecord(ev[2], h->stream));
    }
    return LDPM_OK;
}

int collect_profile(ldpm_ctx *h)
{
    for (auto &pr : h->ev_pairs) {
        float ms = 0;
        CU(cudaEventSynchronize(h->ev_pool[pr[2]]));
        CU(cudaEventElapsedTime(&ms, h->ev_pool[pr[1]], h->ev_pool[pr[2]]));
        h->prof_ms[pr[0]] += ms;
        h->prof_cnt[pr[0]] += 1;
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    h->ev_pairs.clear();
    return LDPM_OK;
}

// Persistent launches of nsteps steps, in chunks of at most 4096 steps (each launch then stays short,
// and the barrier counter, 2 x grid per step, within 32 bits); while profiling each launch is
// bracketed by events (kernel id 5).
int enqueue_persistent(ldpm_ctx *h, int64_t nsteps)
{
    const int64_t grid = std::max(1, h->persist_grid);
    const int64_t cap = std::min<int64_t>(4096, (int64_t)(0xffffffffu / (2 * grid)) - 1);
    for (int64_t left = nsteps; left > 0;) {
        const int64_t len = std::min(left, cap);
        cudaEvent_t a = nullptr, b = nullptr;
        if (h->prof) {
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
                return fail(LDPM_E_CUDA, "event create failed");
            h->ev_pool.push_back(a);
            h->ev_pool.push_back(b);
            h->ev_pairs.push_back({5, (int)h->ev_pool.size() - 2, (int)h->ev_pool.size() - 1});
            CU(cudaEventRecord(a, h->stream));
        }
        int grid_used = 0;
        cudaError_t e = h->prec == LDPM_MIXED ? launch_persistent<float>(h->dm, len, h->pctl, &grid_used, h->stream)
                                              : launch_persistent<double>(h->dm, len, h->pctl, &grid_used, h->stream);
        if (e != cudaSuccess) return fail(LDPM_E_CUDA, "persistent step launch: %s", cudaGetErrorString(e));
        if (h->prof) CU(cudaEventRecord(b, h->stream));
        left -= len;
    }
    return LDPM_OK;
}

// nsteps steps in the handle's launch mode: persistent launches, or launch pairs replayed from CUDA
// graphs captured per chunk length (direct launches while profiling or with graph_chunk < 0).
int enqueue_steps(ldpm_ctx *h, int64_t nsteps)
{
    if (h->launch_mode == LDPM_LAUNCH_PERSISTENT) return enqueue_persistent(h, nsteps);
    if (h->prof) return enqueue_profiled(h, nsteps);
    if (h->graph_chunk < 0) return enqueue_direct(h, nsteps);
    int rc;
    const int64_t chunk = std::max(1, h->graph_chunk);
    for (int64_t left = nsteps; left > 0;) {
        const int64_t len = std::min(left, chunk);
        cudaGraphExec_t ex;
        if ((rc = graph_for(h, len, &ex))) return rc;
        CU(cudaGraphLaunch(ex, h->stream));
        left -= len;
    }
    return LDPM_OK;
}

// Choose the launch mode; the persistent one needs its grid to be co-resident on the device.
int set_launch_mode(ldpm_ctx *h, int mode)
{
    if (mode == LDPM_LAUNCH_PERSISTENT) {
        int grid = 0;
        cudaError_t e = h->prec == LDPM_MIXED ? launch_persistent<float>(h->dm, 0, h->pctl, &grid, h->stream)
                                              : launch_persistent<double>(h->dm, 0, h->pctl, &grid, h->stream);
        if (e != cudaSuccess || grid < 1)
            return fail(LDPM_E_UNSUPPORTED, "persistent launch not possible on this device: %s",
                        cudaGetErrorString(e));
        h->persist_grid = grid;
    }
    h->launch_mode = mode;
    return LDPM_OK;
}

// Run `launch`; while profiling, bracket it with events on the stream (kernel id kid).
template <class Fn>
int timed(ldpm_ctx *h, int kid, Fn &&launch)
{
    if (!h->prof) return launch();
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return fail(LDPM_E_CUDA, "event create failed");
    h->ev_pool.push_back(a);
    h->ev_pool.push_back(b);
    h->ev_pairs.push_back({kid, (int)h->ev_pool.size() - 2, (int)h->ev_pool.size() - 1});
    CU(cudaEventRecord(a, h->stream));
    int rc = launch();
    if (rc) return rc;
    CU(cudaEventRecord(b, h->stream));
    return LDPM_OK;
}

int check_flag(ldpm_ctx *h)
{
    int32_t fl = 0, st = 0;
    CU(cudaMemcpyAsync(&fl, h->dm.flag, sizeof(fl), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&st, h->pctl.status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (st)
        return fail(LDPM_E_TIMEOUT, "a grid barrier of the persistent step kernel waited longer than %.3g s; the "
                    "state is undefined until ldpm_set_state or ldpm_load_checkpoint",
                    1e-9 * (double)h->pctl.wait_ns);
    if (fl) return fail(LDPM_E_UNSTABLE, "non-finite velocity or displacement (time step too large?)");
    return LDPM_OK;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Caller-order state <-> internal arrays.
int download_state(ldpm_ctx *h, std::vector<double> &ps)
{
    ps.resize(16 * (size_t)h->dm.N);
    CU(cudaMemcpyAsync(ps.data(), h->dm.pstate, ps.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return LDPM_OK;
}

// Device scratch of at least n doubles, kept until the handle is destroyed.
int scratch(ldpm_ctx *h, size_t n)
{
    if (h->scratch_n >= n) return LDPM_OK;
    if (h->d_scratch) {
        CU(cudaStreamSynchronize(h->stream));
        cudaFree(h->d_scratch);
        h->d_scratch = nullptr;
        h->scratch_n = 0;
    }
    int rc = dalloc(&h->d_scratch, n);
    if (rc == LDPM_OK) h->scratch_n = n;
    return rc;
}

// ---- per-facet parameters and the adjoint -------------------------------------------------------

// Device allocations released together.
struct DevArena {
    std::vector<void *> ptrs;
    ~DevArena()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    int get(T **p, size_t count)
    {
        int rc = dalloc(p, count);
        if (rc == LDPM_OK) ptrs.push_back(*p);
        return rc;
    }
};

// Byte sizes of the evolving state: everything a step reads and writes.
struct StateBytes {
    size_t ps, pd, pm, hist;
};

StateBytes state_bytes(const ldpm_ctx *h)
{
    StateBytes b;
    b.ps = 16 * (size_t)h->dm.N * sizeof(double);
    b.pd = 8 * (size_t)h->dm.N * sizeof(double);
    b.pm = h->dm.pm32 ? (size_t)kMirror * h->dm.N * sizeof(float) : 0;
    b.hist = 12 * (size_t)h->dm.T * h->r4size();
    return b;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Copy the evolving state to (save) or from (restore) a slot of `total()` bytes.
int state_copy(ldpm_ctx *h, char *slot, bool save)
{
    const StateBytes b = state_bytes(h);
    struct {
        void *dev;
        size_t n;
    } parts[] = {{h->dm.pstate, b.ps}, {h->dm.pdyn, b.pd}, {h->dm.pm32, b.pm}, {h->dm.hist, b.hist}, {h->dm.step, 8}};
    size_t off = 0;
    for (auto &pt : parts) {
        if (pt.n) {
            if (save)
                CU(cudaMemcpyAsync(slot + off, pt.dev, pt.n, cudaMemcpyDeviceToDevice, h->stream));
            else
                CU(cudaMemcpyAsync(pt.dev, slot + off, pt.n, cudaMemcpyDeviceToDevice, h->stream));
        }
        off += align256(pt.n);
    }
    return LDPM_OK;
}

size_t slot_stride(const ldpm_ctx *h)
{
    const StateBytes b = state_bytes(h);
    return align256(b.ps) + align256(b.pd) + align256(b.pm) + align256(b.hist) + 256;
}

template <class R>
int adjoint_run(ldpm_ctx *h, int64_t K, int64_t C, const double *seed, double *J, double *gE0, double *galpha,
                double *gsigma)
{
    const SpecHost &S = h->sp[0];
    const int64_t N = h->dm.N, Fint = 12 * (int64_t)h->dm.T;
    const bool mixed = sizeof(R) == 4;
    int rc;
    // c = -seed / K on constrained DOFs (internal order)
    std::vector<double> c(6 * (size_t)N, 0.0);
    for (int32_t i = 0; i < S.N; ++i) {
        const size_t P = (size_t)S.p0 + S.inv_p[i];
        uint64_t bc;
        std::memcpy(&bc, &h->pconst_h[8 * P + 6], 8);
        for (int d = 0; d < 6; ++d)
            if ((bc >> (8 * d)) & 0xffu) c[6 * P + d] = -seed[6 * (size_t)i + d] / (double)K;
    }
    const int64_t nseg = (K + C - 1) / C;
    const size_t stride = slot_stride(h);
    const size_t rec = mixed ? (size_t)kMirror * N * sizeof(float) : 16 * (size_t)N * sizeof(double);
    const size_t hb = (size_t)Fint * sizeof(R4<R>);
    const size_t snap_stride = align256(rec) + align256(hb);
    DevArena ar;
    char *ckpt = nullptr, *snap = nullptr;
    AdjointModel a;
    for (auto &sp : h->sp) a.reload |= sp.mat.k_t > 0.0;
    if ((rc = ar.get(&ckpt, stride * (size_t)(nseg + 1))) || (rc = ar.get(&snap, snap_stride * (size_t)std::min(C, K))))
        return fail(LDPM_E_OOM, "adjoint: %lld checkpoints of %zu bytes and %lld step snapshots of %zu bytes do "
                                "not fit (use a smaller checkpoint interval)",
                    (long long)(nseg + 1), stride, (long long)std::min(C, K), snap_stride);
    if ((rc = ar.get((double **)&a.cseed, 6 * (size_t)N)) || (rc = ar.get(&a.Qbar, 6 * (size_t)N)) ||
        (rc = ar.get(&a.Ubar, 6 * (size_t)N)) || (rc = ar.get(&a.jacc, (size_t)N)) ||
        (rc = ar.get((R4<R> **)&a.adj_h, (size_t)Fint)) || (rc = ar.get((R4<R> **)&a.gacc, (size_t)Fint)) ||
        (rc = ar.get((R **)&a.tvc2, 4 * (size_t)Fint)))
        return rc;
    if (mixed) {
        if ((rc = ar.get((float **)&a.af, 12 * (size_t)N)) || (rc = ar.get(&a.gsum, 4 * (size_t)Fint))) return rc;
    } else {
        if ((rc = ar.get((double **)&a.af, 8 * (size_t)N))) return rc;
    }
    CU(cudaMemcpyAsync(a.cseed, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemsetAsync(a.jacc, 0, (size_t)N * sizeof(double), h->stream));
    auto fwd = [&](bool objective) -> int {
        int r;
        if ((r = timed(h, 1, [&]() { return launch_facet_any(h, FACET_STEP, nullptr); })) ||
            (r = timed(h, 2, [&]() { return launch_gather_any(h, GATHER_STEP_MID, nullptr); })))
            return r;
        if (objective) CU(launch_objective(h->dm, a, h->stream));
        return LDPM_OK;
    };
    const bool grads = gE0 || galpha || gsigma;
    // n steps from the model's state keeping each step's inputs in slot i: the particle records it
    // reads are copied there, and its history is read from the slot itself.  Slot 0 receives the
    // model's history; step i writes its new history into slot i + 1 (the last step into the model's
    // own buffer), so the history is never copied per step.
    auto run_kept = [&](int64_t n, bool objective) -> int {
        void *own = h->dm.hist;
        CU(cudaMemcpyAsync(snap + align256(rec), own, hb, cudaMemcpyDeviceToDevice, h->stream));
        int r = LDPM_OK;
        for (int64_t i = 0; i < n && r == LDPM_OK; ++i) {
            char *sl = snap + snap_stride * i;
            cudaError_t e = cudaMemcpyAsync(sl, mixed ? (const void *)h->dm.pm32 : (const void *)h->dm.pstate, rec,
                                            cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) {
                r = fail(LDPM_E_CUDA, "adjoint: step input copy: %s", cudaGetErrorString(e));
                break;
            }
            h->dm.hist = sl + align256(rec);
            h->dm.hist_out = i + 1 < n ? (void *)(snap + snap_stride * (i + 1) + align256(rec)) : own;
            r = fwd(objective);
        }
        h->dm.hist = own;
        h->dm.hist_out = nullptr;
        return r;
    };
    // forward sweep: checkpoint at the start of every segment, and the final state.  The last segment
    // is the first one reversed, so its step inputs are kept now instead of being recomputed.
    for (int64_t sg = 0; sg < nseg; ++sg) {
        if ((rc = state_copy(h, ckpt + stride * sg, true))) return rc;
        const int64_t n = std::min(C, K - sg * C);
        if (grads && sg == nseg - 1) {
            if ((rc = run_kept(n, true))) return rc;
        } else {
            for (int64_t i = 0; i < n; ++i)
                if ((rc = fwd(true))) return rc;
        }
    }
    if ((rc = state_copy(h, ckpt + stride * nseg, true))) return rc;
    if ((rc = check_flag(h))) return rc;
    // reverse sweep, segment by segment from the last
    if (grads) {
        CU(launch_adjoint_init<R>(h->dm, a, h->stream));
        for (int64_t sg = nseg - 1; sg >= 0; --sg) {
            const int64_t n = std::min(C, K - sg * C);
            if (sg < nseg - 1) {  // recompute the segment from its checkpoint, keeping each step's inputs
                if ((rc = state_copy(h, ckpt + stride * sg, false))) return rc;
                if ((rc = run_kept(n, false))) return rc;
            }
            for (int64_t i = n - 1; i >= 0; --i) {
                char *sl = snap + snap_stride * i;
                a.snap_p = sl;
                a.snap_h = sl + align256(rec);
                if ((rc = timed(h, 3, [&]() -> int {
                         CU(launch_adjoint_facet<R>(h->dm, a, h->stream));
                         return LDPM_OK;
                     })) ||
                    (rc = timed(h, 4, [&]() -> int {
                         CU(launch_adjoint_gather<R>(h->dm, a, h->stream));
                         return LDPM_OK;
                     })))
                    return rc;
            }
            if (mixed) CU(launch_adjoint_fold<R>(h->dm, a, h->stream));
        }
        if ((rc = state_copy(h, ckpt + stride * nseg, false))) return rc;
    }
    // results
    std::vector<double> jp((size_t)N);
    CU(cudaMemcpyAsync(jp.data(), a.jacc, jp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    std::vector<double> g4(grads ? 4 * (size_t)Fint : 0);
    if (grads)
        CU(cudaMemcpyAsync(g4.data(), mixed ? (const void *)a.gsum : (const void *)a.gacc, g4.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (J) {
        double acc = 0.0;
        for (double x : jp) acc += x;
        *J = acc;
    }
    double *outs[3] = {gE0, galpha, gsigma};
    for (int k3 = 0; k3 < 3; ++k3)
        if (outs[k3])
            for (int32_t k = 0; k < S.F; ++k) outs[k3][k] = g4[4 * (size_t)S.fmap[k] + k3];
    for (int k3 = 0; k3 < 3; ++k3)
        if (outs[k3])
            for (int32_t k = 0; k < S.F; ++k)
                if (!std::isfinite(outs[k3][k])) return fail(LDPM_E_UNSTABLE, "adjoint: non-finite gradient");
    return LDPM_OK;
}

}  // namespace

// =================================================================================================
// C ABI
// =================================================================================================
extern "C" {

const char *ldpm_last_error(void) { return g_err.c_str(); }

int ldpm_create(const ldpm_geometry *geom, const ldpm_material *mat, const ldpm_options *opt, ldpm_t *out)
{
    g_err.clear();
    if (!geom || !mat || !opt) return fail(LDPM_E_INVALID_ARG, "geometry, material and options are required");
    try {
        return create_model(1, geom, mat, opt, out);
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    } catch (...) {
        return fail(LDPM_E_CUDA, "unexpected exception in ldpm_create");
    }
}

int ldpm_step(ldpm_t h, int64_t nsteps)
{
    g_err.clear();
    if (!h || nsteps < 0) return fail(LDPM_E_INVALID_ARG, "bad handle or nsteps < 0");
    if (nsteps == 0) return LDPM_OK;
    DevGuard dg(h->device);
    try {
        return enqueue_steps(h, nsteps);
    } catch (...) {
        return fail(LDPM_E_CUDA, "unexpected exception in ldpm_step");
    }
}

int ldpm_set_launch_mode(ldpm_t h, int32_t mode)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    if (mode != LDPM_LAUNCH_PAIRS && mode != LDPM_LAUNCH_PERSISTENT)
        return fail(LDPM_E_INVALID_ARG, "mode must be LDPM_LAUNCH_PAIRS or LDPM_LAUNCH_PERSISTENT");
    DevGuard dg(h->device);
    return set_launch_mode(h, mode);
}

int32_t ldpm_launch_mode(ldpm_t h)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    return h->launch_mode;
}

int ldpm_set_barrier_wait(ldpm_t h, double seconds, int32_t skip_block)
{
    g_err.clear();
    if (!h || !std::isfinite(seconds) || seconds > 3600.0 || skip_block < -1)
        return fail(LDPM_E_INVALID_ARG, "bad handle, seconds not finite or above 3600, or skip_block < -1");
    h->pctl.wait_ns = seconds > 0 ? (uint64_t)(seconds * 1e9) : 2000000000ull;
    h->pctl.skip_block = skip_block;
    return LDPM_OK;
}

int ldpm_sync(ldpm_t h)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    DevGuard dg(h->device);
    CU(cudaStreamSynchronize(h->stream));
    return check_flag(h);
}

static int get_state_range(ldpm_t h, int s_lo, int s_hi, double *q, double *v, double *hist5, int64_t *step)
{
    DevGuard dg(h->device);
    try {
        // whole-step q_n, v_n from the drifted state; the history is converted and put in the caller's
        // facet order on the device and copied straight into hist5
        const size_t N = (size_t)h->dm.N;
        const int64_t k0 = h->ufoff[s_lo], k1 = h->ufoff[s_hi];
        int rc;
        if ((rc = scratch(h, 12 * N + (hist5 ? 5 * (size_t)(k1 - k0) : 0)))) return rc;
        double *d12 = h->d_scratch, *d5 = h->d_scratch + 12 * N;
        std::vector<double> qv(12 * N);
        CU(launch_unkick(h->dm, d12, h->stream));
        CU(cudaMemcpyAsync(qv.data(), d12, qv.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (hist5) {
            CU(h->prec == LDPM_MIXED ? launch_hist_to_user<float>(h->dm, h->d_umap + k0, k1 - k0, d5, h->stream)
                                     : launch_hist_to_user<double>(h->dm, h->d_umap + k0, k1 - k0, d5, h->stream));
            CU(cudaMemcpyAsync(hist5, d5, 5 * (size_t)(k1 - k0) * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
        }
        int64_t st = 0;
        CU(cudaMemcpyAsync(&st, h->dm.step, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        size_t base_p = 0;
        for (int si = s_lo; si < s_hi; ++si) {
            const SpecHost &S = h->sp[si];
            for (int32_t i = 0; i < S.N; ++i) {
                const size_t P = (size_t)S.p0 + S.inv_p[i];
                for (int k = 0; k < 6; ++k) {
                    if (q) q[6 * (base_p + i) + k] = qv[12 * P + k];
                    if (v) v[6 * (base_p + i) + k] = qv[12 * P + 6 + k];
                }
            }
            base_p += S.N;
        }
        if (step) *step = st;
        return check_flag(h);
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    }
}

int ldpm_get_state(ldpm_t h, double *q, double *v, double *hist5, int64_t *step)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    return get_state_range(h, 0, (int)h->sp.size(), q, v, hist5, step);
}

int ldpm_get_state_device(ldpm_t h, double *q, double *v, double *hist5, int64_t *step)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    DevGuard dg(h->device);
    CU(launch_state_to_user(h->dm, h->d_pmap, h->dm.N, q, v, h->stream));
    if (hist5) {
        const int64_t nf = h->ufoff.back();
        CU(h->prec == LDPM_MIXED ? launch_hist_to_user<float>(h->dm, h->d_umap, nf, hist5, h->stream)
                                 : launch_hist_to_user<double>(h->dm, h->d_umap, nf, hist5, h->stream));
    }
    if (step) CU(cudaMemcpyAsync(step, h->dm.step, sizeof(int64_t), cudaMemcpyDeviceToDevice, h->stream));
    return LDPM_OK;
}

int ldpm_set_state(ldpm_t h, const double *q, const double *v, const double *hist5, int64_t step)
{
    g_err.clear();
    if (!h || !q || !v) return fail(LDPM_E_INVALID_ARG, "bad handle or NULL q/v");
    if (h->sp.size() != 1) return fail(LDPM_E_INVALID_ARG, "ldpm_set_state applies to single-specimen handles");
    DevGuard dg(h->device);
    try {
        std::vector<double> ps;
        int rc = download_state(h, ps);
        if (rc) return rc;
        const int64_t Fint = 12 * (int64_t)h->dm.T;
        std::vector<double> h5(5 * (size_t)Fint, 0.0);
        size_t base_p = 0, base_f = 0;
        for (auto &S : h->sp) {
            S.W_kin0 = 0.0;
            for (int32_t i = 0; i < S.N; ++i) {
                const size_t P = (size_t)S.p0 + S.inv_p[i];
                for (int k = 0; k < 6; ++k) {
                    ps[16 * P + 3 + k] = q[6 * (base_p + i) + k];
                    const double vv = v[6 * (base_p + i) + k];
                    ps[16 * P + 9 + k] = vv;
                    S.W_kin0 += 0.5 * vv * vv / h->inv_mass[6 * P + k];
                }
            }
            if (hist5)
                for (int32_t k = 0; k < S.F; ++k) {
                    double *dst = &h5[5 * (size_t)S.fmap[k]];
                    const double *src = hist5 + 5 * (base_f + k);
                    const double sg = S.fswap[k] ? -1.0 : 1.0;
                    dst[0] = src[0];
                    dst[1] = sg * src[1];
                    dst[2] = sg * src[2];
                    dst[3] = sg * src[3];
                    dst[4] = src[4];
                }
            base_p += S.N;
            base_f += S.F;
        }
        CU(cudaMemcpy(h->dm.pstate, ps.data(), ps.size() * sizeof(double), cudaMemcpyHostToDevice));
        CU(launch_mirror(h->dm, h->stream));
        CU(cudaMemset(h->dm.pdyn, 0, 8 * (size_t)h->dm.N * sizeof(double)));
        double *d5 = nullptr;
        if ((rc = dalloc(&d5, 5 * (size_t)Fint))) return rc;
        cudaError_t e = cudaMemcpy(d5, h5.data(), h5.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = h->prec == LDPM_MIXED ? launch_hist_from_user<float>(h->dm, d5, h->stream)
                                      : launch_hist_from_user<double>(h->dm, d5, h->stream);
        cudaError_t e2 = cudaStreamSynchronize(h->stream);
        cudaFree(d5);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(LDPM_E_CUDA, "history upload: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        CU(cudaMemcpy(h->dm.step, &step, sizeof(step), cudaMemcpyHostToDevice));
        CU(cudaMemset(h->dm.flag, 0, sizeof(int32_t)));
        CU(cudaMemset(h->pctl.status, 0, sizeof(int32_t)));
        if ((rc = forces_from_history(h))) return rc;
        if ((rc = kick(h))) return rc;
        CU(cudaStreamSynchronize(h->stream));
        return LDPM_OK;
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    }
}

static int energy_of(ldpm_t h, int s, double out[4], double reaction[12])
{
    const SpecHost &S = h->sp[s];
    cudaError_t e = launch_energy(h->dm, S.p0, S.p0 + S.N, h->d_partial, h->d_ticket, h->d_out16, h->stream);
    if (e != cudaSuccess) return fail(LDPM_E_CUDA, "energy launch: %s", cudaGetErrorString(e));
    CU(cudaMemcpyAsync(h->h_out16, h->d_out16, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    const double *r = h->h_out16;
    const double Wint = r[0], Wext = r[1], Wkin = r[2];
    if (out) {
        out[0] = Wext;
        out[1] = Wint;
        out[2] = Wkin;
        const double den = std::fabs(Wext) + S.W_kin0;
        out[3] = den > 0 ? 100.0 * std::fabs(Wext + S.W_kin0 - Wint - Wkin) / den : 0.0;
    }
    if (reaction)
        for (int k = 0; k < 12; ++k) reaction[k] = r[4 + k];
    return LDPM_OK;
}

int ldpm_energy(ldpm_t h, double out[4], double reaction[12])
{
    g_err.clear();
    if (!h || !out) return fail(LDPM_E_INVALID_ARG, "bad handle or NULL out");
    if (h->sp.size() != 1) return fail(LDPM_E_INVALID_ARG, "batch handle: use ldpm_batch_energy");
    DevGuard dg(h->device);
    int rc = energy_of(h, 0, out, reaction);
    if (rc) return rc;
    return check_flag(h);
}

int ldpm_facet_forces(ldpm_t h, double *F3, double *f6)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    DevGuard dg(h->device);
    try {
        // per-facet forces are not kept by the step; rebuild them from the stored tractions (this
        // rewrites the per-vertex shares with the same values)
        int rc = launch_facet_any(h, FACET_FROM_HIST, nullptr);
        if (rc) return rc;
        CU(cudaStreamSynchronize(h->stream));
        const int64_t Fint = 12 * (int64_t)h->dm.T;
        std::vector<double> fo(4 * (size_t)Fint), pd(8 * (size_t)h->dm.N);
        if (h->prec == LDPM_MIXED) {
            std::vector<float4> t(Fint);
            CU(cudaMemcpy(t.data(), h->dm.fout, Fint * sizeof(float4), cudaMemcpyDeviceToHost));
            for (int64_t f = 0; f < Fint; ++f) {
                fo[4 * f] = t[f].x;
                fo[4 * f + 1] = t[f].y;
                fo[4 * f + 2] = t[f].z;
            }
        } else {
            CU(cudaMemcpy(fo.data(), h->dm.fout, Fint * 4 * sizeof(double), cudaMemcpyDeviceToHost));
        }
        CU(cudaMemcpy(pd.data(), h->dm.pdyn, pd.size() * sizeof(double), cudaMemcpyDeviceToHost));
        size_t base_p = 0, base_f = 0;
        for (auto &S : h->sp) {
            if (F3)
                for (int32_t k = 0; k < S.F; ++k) {
                    const double sg = S.fswap[k] ? -1.0 : 1.0;
                    for (int a = 0; a < 3; ++a) F3[3 * (base_f + k) + a] = sg * fo[4 * (size_t)S.fmap[k] + a];
                }
            if (f6)
                for (int32_t i = 0; i < S.N; ++i) {
                    const size_t P = (size_t)S.p0 + S.inv_p[i];
                    for (int k = 0; k < 6; ++k) f6[6 * (base_p + i) + k] = pd[8 * P + k];
                }
            base_p += S.N;
            base_f += S.F;
        }
        return LDPM_OK;
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    }
}

static int metrics_range(ldpm_t h, int s_lo, int s_hi, double *crack_opening, double *tet_volumetric_strain)
{
    DevGuard dg(h->device);
    try {
        int rc = launch_facet_any(h, FACET_METRIC, nullptr);
        if (rc) return rc;
        CU(cudaStreamSynchronize(h->stream));
        const int64_t Fint = 12 * (int64_t)h->dm.T;
        std::vector<double> fo(4 * (size_t)Fint);
        if (h->prec == LDPM_MIXED) {
            std::vector<float4> t(Fint);
            CU(cudaMemcpy(t.data(), h->dm.fout, Fint * sizeof(float4), cudaMemcpyDeviceToHost));
            for (int64_t f = 0; f < Fint; ++f) {
                fo[4 * f] = t[f].x;
                fo[4 * f + 1] = t[f].y;
            }
        } else {
            CU(cudaMemcpy(fo.data(), h->dm.fout, Fint * 4 * sizeof(double), cudaMemcpyDeviceToHost));
        }
        size_t base_f = 0, base_t = 0;
        for (int si = s_lo; si < s_hi; ++si) {
            const SpecHost &S = h->sp[si];
            if (crack_opening)
                for (int32_t k = 0; k < S.F; ++k) crack_opening[base_f + k] = fo[4 * (size_t)S.fmap[k]];
            if (tet_volumetric_strain)
                for (int32_t t = 0; t < S.T; ++t) tet_volumetric_strain[base_t + t] = fo[4 * (12 * (size_t)S.tmap[t]) + 1];
            base_f += S.F;
            base_t += S.T;
        }
        return LDPM_OK;
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    }
}

int ldpm_metrics(ldpm_t h, double *crack_opening, double *tet_volumetric_strain)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    return metrics_range(h, 0, (int)h->sp.size(), crack_opening, tet_volumetric_strain);
}

int ldpm_set_bc(ldpm_t h, const int32_t *mask, const double *vel, double ramp_time)
{
    g_err.clear();
    if (!h || !mask || !std::isfinite(ramp_time)) return fail(LDPM_E_INVALID_ARG, "bad handle, mask or ramp_time");
    if (h->sp.size() != 1) return fail(LDPM_E_INVALID_ARG, "ldpm_set_bc applies to single-specimen handles");
    DevGuard dg(h->device);
    SpecHost &S = h->sp[0];
    std::vector<double> bv(6 * (size_t)h->dm.N, 0.0), bm(6 * (size_t)h->dm.N, 0.0);
    for (int32_t i = 0; i < S.N; ++i) {
        const size_t P = (size_t)S.p0 + S.inv_p[i];
        uint64_t bits = 0;
        for (int k = 0; k < 6; ++k) {
            const int mk = mask[6 * (size_t)i + k];
            if (mk < 0 || mk > 2) return fail(LDPM_E_INVALID_ARG, "bc mask must be 0, 1 or 2");
            bits |= (uint64_t)mk << (8 * k);
            bv[6 * P + k] = vel ? vel[6 * (size_t)i + k] : 0.0;
            bm[6 * P + k] = bv[6 * P + k] / h->inv_mass[6 * P + k];
        }
        std::memcpy(&h->pconst_h[8 * P + 6], &bits, 8);
    }
    S.ramp_time = ramp_time;
    // back to the whole-step state under the old conditions, then forward under the new ones
    CU(launch_unkick(h->dm, nullptr, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaMemcpy(h->dm.pconst, h->pconst_h.data(), h->pconst_h.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->dm.bc_vel, bv.data(), bv.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->dm.bc_vm, bm.data(), bm.size() * sizeof(double), cudaMemcpyHostToDevice));
    int rc = update_law(h);
    if (rc) return rc;
    if ((rc = kick(h))) return rc;
    CU(cudaStreamSynchronize(h->stream));
    return LDPM_OK;
}

int ldpm_info(ldpm_t h, int64_t info[5], double *dt)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    DevGuard dg(h->device);
    int64_t N = 0, T = 0, F = 0;
    for (auto &S : h->sp) {
        N += S.N;
        T += S.T;
        F += S.F;
    }
    if (info) {
        CU(cudaStreamSynchronize(h->stream));
        int64_t st = 0;
        CU(cudaMemcpy(&st, h->dm.step, sizeof(st), cudaMemcpyDeviceToHost));
        info[0] = N;
        info[1] = T;
        info[2] = F;
        info[3] = h->prec;
        info[4] = st;
    }
    if (dt) *dt = h->sp[0].dt;
    return LDPM_OK;
}

int ldpm_profile(ldpm_t h, int32_t enable)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    DevGuard dg(h->device);
    if (h->prof) collect_profile(h);
    h->prof = enable != 0;
    for (int k = 0; k < 6; ++k) {
        h->prof_ms[k] = 0;
        h->prof_cnt[k] = 0;
    }
    return LDPM_OK;
}

int ldpm_profile_read(ldpm_t h, double *ms, int64_t *count, int32_t n)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    DevGuard dg(h->device);
    int rc = collect_profile(h);
    if (rc) return rc;
    for (int k = 0; k < n && k < 6; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (count) count[k] = h->prof_cnt[k];
    }
    return LDPM_OK;
}

int64_t ldpm_checkpoint_size(ldpm_t h)
{
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    const int64_t Fint = 12 * (int64_t)h->dm.T;
    return (int64_t)(16 + 8) * h->dm.N * 8 + Fint * (int64_t)h->r4size() + 8 + 8 + 8 * (int64_t)h->sp.size();
}

int ldpm_save_checkpoint(ldpm_t h, void *buf)
{
    g_err.clear();
    if (!h || !buf) return fail(LDPM_E_INVALID_ARG, "bad handle or NULL buffer");
    DevGuard dg(h->device);
    char *p = static_cast<char *>(buf);
    const size_t n_ps = 16 * (size_t)h->dm.N * 8, n_pd = 8 * (size_t)h->dm.N * 8;
    const size_t n_h = 12 * (size_t)h->dm.T * h->r4size();
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaMemcpy(p, h->dm.pstate, n_ps, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(p + n_ps, h->dm.pdyn, n_pd, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(p + n_ps + n_pd, h->dm.hist, n_h, cudaMemcpyDeviceToHost));
    char *q = p + n_ps + n_pd + n_h;
    CU(cudaMemcpy(q, h->dm.step, 8, cudaMemcpyDeviceToHost));
    int32_t fl = 0;
    CU(cudaMemcpy(&fl, h->dm.flag, 4, cudaMemcpyDeviceToHost));
    int64_t fl64 = fl;
    std::memcpy(q + 8, &fl64, 8);
    for (size_t s = 0; s < h->sp.size(); ++s) std::memcpy(q + 16 + 8 * s, &h->sp[s].W_kin0, 8);
    return LDPM_OK;
}

int ldpm_load_checkpoint(ldpm_t h, const void *buf)
{
    g_err.clear();
    if (!h || !buf) return fail(LDPM_E_INVALID_ARG, "bad handle or NULL buffer");
    DevGuard dg(h->device);
    const char *p = static_cast<const char *>(buf);
    const size_t n_ps = 16 * (size_t)h->dm.N * 8, n_pd = 8 * (size_t)h->dm.N * 8;
    const size_t n_h = 12 * (size_t)h->dm.T * h->r4size();
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaMemcpy(h->dm.pstate, p, n_ps, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->dm.pdyn, p + n_ps, n_pd, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->dm.hist, p + n_ps + n_pd, n_h, cudaMemcpyHostToDevice));
    const char *q = p + n_ps + n_pd + n_h;
    CU(cudaMemcpy(h->dm.step, q, 8, cudaMemcpyHostToDevice));
    int64_t fl64;
    std::memcpy(&fl64, q + 8, 8);
    int32_t fl = (int32_t)fl64;
    CU(cudaMemcpy(h->dm.flag, &fl, 4, cudaMemcpyHostToDevice));
    CU(cudaMemset(h->pctl.status, 0, sizeof(int32_t)));
    for (size_t s = 0; s < h->sp.size(); ++s) std::memcpy(&h->sp[s].W_kin0, q + 16 + 8 * s, 8);
    CU(launch_mirror(h->dm, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return LDPM_OK;
}

int ldpm_batch_create(int32_t n, const ldpm_geometry *geoms, const ldpm_material *mats, const ldpm_options *opts,
                      ldpm_t *out)
{
    g_err.clear();
    if (n < 1 || !geoms || !mats || !opts) return fail(LDPM_E_INVALID_ARG, "need n >= 1 and non-NULL arrays");
    try {
        return create_model(n, geoms, mats, opts, out);
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    } catch (...) {
        return fail(LDPM_E_CUDA, "unexpected exception in ldpm_batch_create");
    }
}

int ldpm_batch_step(ldpm_t h, int64_t nsteps) { return ldpm_step(h, nsteps); }

int32_t ldpm_batch_size(ldpm_t h)
{
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    return (int32_t)h->sp.size();
}

int ldpm_batch_get_state(ldpm_t h, int32_t idx, double *q, double *v, double *hist5, int64_t *step)
{
    g_err.clear();
    if (!h || idx < 0 || idx >= (int32_t)h->sp.size()) return fail(LDPM_E_INVALID_ARG, "bad handle or index");
    return get_state_range(h, idx, idx + 1, q, v, hist5, step);
}

int ldpm_batch_energy(ldpm_t h, int32_t idx, double out[4], double reaction[12])
{
    g_err.clear();
    if (!h || !out || idx < 0 || idx >= (int32_t)h->sp.size())
        return fail(LDPM_E_INVALID_ARG, "bad handle, index or NULL out");
    DevGuard dg(h->device);
    int rc = energy_of(h, idx, out, reaction);
    if (rc) return rc;
    return check_flag(h);
}

int ldpm_batch_metrics(ldpm_t h, int32_t idx, double *crack_opening, double *tet_volumetric_strain)
{
    g_err.clear();
    if (!h || idx < 0 || idx >= (int32_t)h->sp.size()) return fail(LDPM_E_INVALID_ARG, "bad handle or index");
    return metrics_range(h, idx, idx + 1, crack_opening, tet_volumetric_strain);
}

int ldpm_batch_info(ldpm_t h, int32_t idx, int64_t info[5], double *dt)
{
    g_err.clear();
    if (!h || idx < 0 || idx >= (int32_t)h->sp.size()) return fail(LDPM_E_INVALID_ARG, "bad handle or index");
    DevGuard dg(h->device);
    const SpecHost &S = h->sp[idx];
    if (info) {
        CU(cudaStreamSynchronize(h->stream));
        int64_t st = 0;
        CU(cudaMemcpy(&st, h->dm.step, sizeof(st), cudaMemcpyDeviceToHost));
        info[0] = S.N;
        info[1] = S.T;
        info[2] = S.F;
        info[3] = h->prec;
        info[4] = st;
    }
    if (dt) *dt = S.dt;
    return LDPM_OK;
}

int ldpm_perturb(ldpm_t h, const double *dq)
{
    g_err.clear();
    if (!h || !dq) return fail(LDPM_E_INVALID_ARG, "bad handle or NULL dq");
    DevGuard dg(h->device);
    try {
        std::vector<double> di(6 * (size_t)h->dm.N, 0.0);
        size_t base = 0;
        for (auto &S : h->sp) {
            for (int32_t i = 0; i < S.N; ++i) {
                const size_t P = (size_t)S.p0 + S.inv_p[i];
                for (int k = 0; k < 6; ++k) {
                    const double x = dq[6 * (base + i) + k];
                    if (!std::isfinite(x)) return fail(LDPM_E_INVALID_ARG, "dq is not finite");
                    di[6 * P + k] = x;
                }
            }
            base += S.N;
        }
        DevArena ar;
        double *d = nullptr;
        int rc;
        if ((rc = ar.get(&d, di.size()))) return rc;
        CU(cudaMemcpyAsync(d, di.data(), di.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CU(launch_perturb(h->dm, d, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        return LDPM_OK;
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    }
}

int ldpm_set_facet_params(ldpm_t h, const double *E0, const double *alpha, const double *sigma_t)
{
    g_err.clear();
    if (!h) return fail(LDPM_E_INVALID_ARG, "bad handle");
    if (h->sp.size() != 1) return fail(LDPM_E_INVALID_ARG, "per-facet parameters take a single-specimen model");
    DevGuard dg(h->device);
    try {
        const SpecHost &S = h->sp[0];
        const int64_t Fint = 12 * (int64_t)h->dm.T;
        const double *src[3] = {E0, alpha, sigma_t};
        const double mat[3] = {S.mat.E0, S.mat.alpha, S.mat.sigma_t};
        for (int k3 = 0; k3 < 3; ++k3)
            if (src[k3])
                for (int32_t k = 0; k < S.F; ++k)
                    if (!(std::isfinite(src[k3][k]) && src[k3][k] > 0.0))
                        return fail(LDPM_E_INVALID_ARG, "per-facet parameter %d of facet %d is not finite and > 0", k3, k);
        CU(cudaStreamSynchronize(h->stream));
        for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);  // captured launches hold the old model
        h->graphs.clear();
        if (!E0 && !alpha && !sigma_t) {
            if (h->dm.pf) cudaFree(h->dm.pf);
            h->dm.pf = nullptr;
            return LDPM_OK;
        }
        std::vector<double> v(4 * (size_t)Fint, 0.0);
        for (int64_t f = 0; f < Fint; ++f)
            for (int k3 = 0; k3 < 3; ++k3) v[4 * f + k3] = mat[k3];
        for (int k3 = 0; k3 < 3; ++k3)
            if (src[k3])
                for (int32_t k = 0; k < S.F; ++k) v[4 * (size_t)S.fmap[k] + k3] = src[k3][k];
        if (!h->dm.pf) {
            int rc = h->prec == LDPM_MIXED ? dalloc((float4 **)&h->dm.pf, (size_t)Fint)
                                           : dalloc((double4a **)&h->dm.pf, (size_t)Fint);
            if (rc) return rc;
        }
        if (h->prec == LDPM_MIXED) {
            std::vector<float> f32(v.begin(), v.end());
            CU(cudaMemcpy(h->dm.pf, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice));
        } else {
            CU(cudaMemcpy(h->dm.pf, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
        return LDPM_OK;
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    }
}

int ldpm_adjoint(ldpm_t h, int64_t nsteps, int32_t ckpt_every, const double *seed, double *J, double *gE0,
                 double *galpha, double *gsigma_t)
{
    g_err.clear();
    if (!h || nsteps < 1 || ckpt_every < 1 || !seed)
        return fail(LDPM_E_INVALID_ARG, "bad handle, nsteps < 1, ckpt_every < 1 or NULL seed");
    if (h->sp.size() != 1) return fail(LDPM_E_INVALID_ARG, "the adjoint takes a single-specimen model");
    DevGuard dg(h->device);
    try {
        CU(cudaStreamSynchronize(h->stream));
        return h->prec == LDPM_MIXED ? adjoint_run<float>(h, nsteps, ckpt_every, seed, J, gE0, galpha, gsigma_t)
                                     : adjoint_run<double>(h, nsteps, ckpt_every, seed, J, gE0, galpha, gsigma_t);
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    } catch (...) {
        return fail(LDPM_E_CUDA, "unexpected exception in ldpm_adjoint");
    }
}

int ldpm_facet_law_vjp(int32_t precision, const ldpm_material *mat, int64_t n, const double *in, const double *adj_out,
                       double *out, double *adj_in)
{
    g_err.clear();
    if (!mat || n < 0 || (n > 0 && (!in || !adj_out || !out || !adj_in)) ||
        (precision != LDPM_FP64 && precision != LDPM_MIXED))
        return fail(LDPM_E_INVALID_ARG, "bad precision, material, count or NULL buffer");
    int rc = check_material(*mat);
    if (rc) return rc;
    if (n == 0) return LDPM_OK;
    try {
        DevArena ar;
        double *d_in, *d_ao, *d_out, *d_ai;
        if ((rc = ar.get(&d_in, 16 * (size_t)n)) || (rc = ar.get(&d_ao, 4 * (size_t)n)) ||
            (rc = ar.get(&d_out, 4 * (size_t)n)) || (rc = ar.get(&d_ai, 16 * (size_t)n)))
            return rc;
        CU(cudaMemcpy(d_in, in, 16 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(d_ao, adj_out, 4 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice));
        cudaError_t e;
        if (precision == LDPM_MIXED) {
            LawConst<float> c, *dc;
            law_const<float>(*mat, 0.0, c);
            if ((rc = ar.get(&dc, 1))) return rc;
            CU(cudaMemcpy(dc, &c, sizeof(c), cudaMemcpyHostToDevice));
            e = launch_law_vjp<float>(dc, n, d_in, d_ao, d_out, d_ai, 0);
        } else {
            LawConst<double> c, *dc;
            law_const<double>(*mat, 0.0, c);
            if ((rc = ar.get(&dc, 1))) return rc;
            CU(cudaMemcpy(dc, &c, sizeof(c), cudaMemcpyHostToDevice));
            e = launch_law_vjp<double>(dc, n, d_in, d_ao, d_out, d_ai, 0);
        }
        if (e != cudaSuccess) return fail(LDPM_E_CUDA, "law VJP launch: %s", cudaGetErrorString(e));
        CU(cudaDeviceSynchronize());
        CU(cudaMemcpy(out, d_out, 4 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(adj_in, d_ai, 16 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));
        return LDPM_OK;
    } catch (const std::bad_alloc &) {
        return fail(LDPM_E_OOM, "host allocation failed");
    }
}

int ldpm_launch_shape(ldpm_t h, int32_t shape[2])
{
    g_err.clear();
    if (!h || !shape) return fail(LDPM_E_INVALID_ARG, "bad handle or NULL shape");
    shape[0] = h->dm.tets_per_block;
    shape[1] = h->dm.gather_lanes;
    return LDPM_OK;
}

void ldpm_destroy(ldpm_t h)
{
    if (!h) return;
    {
        DevGuard dg(h->device);
        if (h->stream) cudaStreamSynchronize(h->stream);
        free_model(h);
    }
    delete h;
}

}  // extern "C"
