// hf_api.cu -- C ABI of the Hirsch-Fye QMC / RDMFT library (declared in include/hf.h).
//
// Host side of one context: validates parameters, builds the trapped lattice of eq. 1 (square,
// disc, box or slab) and its point-group orbits, lays the device state out inside the caller's
// workspace and sequences the kernels of one RDMFT iteration ("Model and Methods": lattice step
// per Matsubara frequency, one impurity problem per inequivalent site, many Markov chains per
// impurity).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>
#include <algorithm>
#include <chrono>
#include <tuple>

#include "hf_internal.cuh"
#include "k_lattice.cuh"
#include "k_refresh_tc.cuh"

namespace {

thread_local std::string g_init_error;

// ---------------------------------------------------------------------------------------
// Lattice of eq. 1: sites, trap potential V_i = V0 r_i^2, nearest-neighbour hopping t.
//   geometry 0: Lx x Ly square, site (x, y) -> y Lx + x, centre ((Lx-1)/2, (Ly-1)/2).
//   geometry 1: site-centred disc x^2 + y^2 <= R^2 (R = Lx) in row order (y, then x).
//   geometry 2: Lx x Ly x Lz box, site (x, y, z) -> (z Ly + y) Lx + x, spherical trap
//               V0 (dx^2 + dy^2 + dz^2) about the box centre; periodic = 1 wraps all three axes.
//   geometry 3: slab of Lz layers, same numbering, cylindrical trap V0 (dx^2 + dy^2) (the
//               component perpendicular to the slab dropped), always periodic across the layers;
//               periodic = 1 also wraps x and y.  ("Efficient simulations for three dimensions".)
// With periodic boundaries the trap is measured from the box centre, so a wrapped bond joins two
// sites of equal potential.
// Orbits: the point operations about the trap centre that map the site set onto itself --
// (dx, dy) -> (+-dx, +-dy), (+-dy, +-dx) in two dimensions, the 48 signed axis permutations for
// the box, and for the slab the 8 in-plane ones combined with z -> +-z + c (mod Lz), the layers
// being equivalent.  The representative of an orbit is its smallest site index, inequivalent
// sites are numbered by increasing representative; a site whose sublattice parity differs from
// its representative's carries the spin exchange of an antiferromagnetic state.
// Band order: the lattice step factors H0 as a band matrix, so sites are placed along the band
// (order / pos) with every periodic axis folded (0, n-1, 1, n-2, ...): a wrapped bond then spans
// at most two positions along its axis instead of n - 1.  The slab's layers come innermost.
// ---------------------------------------------------------------------------------------
struct HostLattice {
    int N = 0;
    int b = 0;                      // band half-width of H0 in the band order
    std::vector<int> x, y, zc;      // integer coordinates (zc = 0 in two dimensions)
    std::vector<double> dx, dy, dz, V;
    std::vector<int> parity, z;     // sublattice parity (+-1), number of neighbours
    std::vector<std::vector<int>> nbr;
    std::vector<int> rep, rep_of, flip, site_rep;
    std::vector<int> order, pos;    // band position -> site, site -> band position
    std::vector<int> gdn;           // image of each site under an operation that exchanges the
                                    // sublattices (empty if the group has none)
};

// Position of coordinate c (0 <= c < n) along a folded periodic axis: 0, n-1, 1, n-2, ...
int fold(int c, int n) { return 2 * c < n ? 2 * c : 2 * (n - 1 - c) + 1; }

bool build_lattice(const hf_params& p, HostLattice& lat, std::string& err) {
    std::map<std::tuple<int, int, int>, int> index;
    const int g = p.geometry;
    const bool three_d = (g == 2 || g == 3);
    const int Lz = three_d ? p.Lz : 1;
    double cx = 0.0, cy = 0.0, cz = 0.0;
    if (g == 0 || three_d) {
        if (p.Lx < 1 || p.Ly < 1 || Lz < 1) { err = "Lx, Ly (and Lz) must be >= 1"; return false; }
        const bool wrap_xy = p.periodic != 0 && three_d;
        const bool wrap_z = (g == 3) || (g == 2 && p.periodic != 0);
        if ((wrap_xy && (p.Lx % 2 || p.Lx < 4 || p.Ly % 2 || p.Ly < 4)) ||
            (wrap_z && (Lz % 2 || Lz < 4))) {
            err = "a periodic axis of the box or slab needs an even length >= 4";
            return false;
        }
        for (int zz = 0; zz < Lz; ++zz)
            for (int yy = 0; yy < p.Ly; ++yy)
                for (int xx = 0; xx < p.Lx; ++xx) {
                    lat.x.push_back(xx); lat.y.push_back(yy); lat.zc.push_back(zz);
                }
        cx = (p.Lx - 1) / 2.0;
        cy = (p.Ly - 1) / 2.0;
        cz = (Lz - 1) / 2.0;
    } else if (g == 1) {
        const int R = p.Lx;
        if (R < 0) { err = "disc radius must be >= 0"; return false; }
        for (int yy = -R; yy <= R; ++yy)
            for (int xx = -R; xx <= R; ++xx)
                if (xx * xx + yy * yy <= R * R) {
                    lat.x.push_back(xx); lat.y.push_back(yy); lat.zc.push_back(0);
                }
    } else {
        err = "geometry must be 0 (square), 1 (disc), 2 (box) or 3 (slab)";
        return false;
    }
    lat.N = static_cast<int>(lat.x.size());
    const int N = lat.N;
    for (int i = 0; i < N; ++i) index[{lat.x[i], lat.y[i], lat.zc[i]}] = i;
    lat.dx.resize(N); lat.dy.resize(N); lat.dz.resize(N); lat.V.resize(N);
    lat.parity.resize(N); lat.z.resize(N);
    lat.nbr.assign(N, {});
    const bool wx = p.periodic != 0 && (g == 0 || three_d);   // wrapped axes
    const bool wz = (g == 3) || (g == 2 && p.periodic != 0);
    const int n_off = three_d ? 6 : 4;
    const int off[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (int i = 0; i < N; ++i) {
        lat.dx[i] = lat.x[i] - cx;
        lat.dy[i] = lat.y[i] - cy;
        lat.dz[i] = three_d ? lat.zc[i] - cz : 0.0;
        const double r2z = (g == 2) ? lat.dz[i] * lat.dz[i] : 0.0;
        lat.V[i] = p.V0 * (lat.dx[i] * lat.dx[i] + lat.dy[i] * lat.dy[i] + r2z);
        lat.parity[i] = (((lat.x[i] + lat.y[i] + lat.zc[i]) % 2) + 2) % 2 == 0 ? 1 : -1;
        for (int o = 0; o < n_off; ++o) {
            int xn = lat.x[i] + off[o][0], yn = lat.y[i] + off[o][1], zn = lat.zc[i] + off[o][2];
            if (wx) {
                xn = ((xn % p.Lx) + p.Lx) % p.Lx;
                yn = ((yn % p.Ly) + p.Ly) % p.Ly;
            }
            if (wz) zn = ((zn % Lz) + Lz) % Lz;
            auto it = index.find({xn, yn, zn});
            if (it != index.end() && it->second != i) {
                bool dup = false;
                for (int j : lat.nbr[i]) dup |= (j == it->second);
                if (!dup) lat.nbr[i].push_back(it->second);
            }
        }
        lat.z[i] = static_cast<int>(lat.nbr[i].size());
    }
    // band order
    lat.pos.resize(N);
    lat.order.resize(N);
    for (int i = 0; i < N; ++i) {
        const int px = wx ? fold(lat.x[i], p.Lx) : lat.x[i];
        const int py = wx ? fold(lat.y[i], p.Ly) : lat.y[i];
        int k = i;                                               // disc: row order
        if (g == 0) k = py * p.Lx + px;
        if (g == 2) k = ((wz ? fold(lat.zc[i], Lz) : lat.zc[i]) * p.Ly + py) * p.Lx + px;
        if (g == 3) k = (py * p.Lx + px) * Lz + fold(lat.zc[i], Lz);
        lat.pos[i] = k;
        lat.order[k] = i;
    }
    for (int i = 0; i < N; ++i)
        for (int j : lat.nbr[i]) lat.b = std::max(lat.b, std::abs(lat.pos[j] - lat.pos[i]));
    // orbits: operations d -> (sgn_a d[perm_a]) about the centre; for the slab the layer index
    // maps as z -> (sgn_z z + shift) mod Lz instead
    struct Op { int perm[3]; int sgn[3]; int shift; };
    std::vector<Op> ops;
    const int perms[6][3] = {{0, 1, 2}, {1, 0, 2}, {0, 2, 1}, {2, 1, 0}, {1, 2, 0}, {2, 0, 1}};
    const int n_perm = (g == 2) ? 6 : 2;
    const int n_shift = (g == 3) ? Lz : 1;
    for (int pi = 0; pi < n_perm; ++pi)
        for (int sx = 1; sx >= -1; sx -= 2)
            for (int sy = 1; sy >= -1; sy -= 2)
                for (int sz = 1; sz >= (three_d ? -1 : 1); sz -= 2)
                    for (int c = 0; c < n_shift; ++c) {
                        Op op{};
                        for (int a = 0; a < 3; ++a) op.perm[a] = perms[pi][a];
                        op.sgn[0] = sx; op.sgn[1] = sy; op.sgn[2] = sz;
                        op.shift = c;
                        ops.push_back(op);
                    }
    std::vector<std::vector<int>> images;
    for (const Op& op : ops) {
        std::vector<int> img(N);
        bool ok = true;
        for (int i = 0; i < N && ok; ++i) {
            const double d[3] = {lat.dx[i], lat.dy[i], lat.dz[i]};
            const double xf = op.sgn[0] * d[op.perm[0]] + cx;
            const double yf = op.sgn[1] * d[op.perm[1]] + cy;
            const long xi = std::lround(xf), yi = std::lround(yf);
            long zi = 0;
            if (g == 3) {
                zi = ((op.sgn[2] * lat.zc[i] + op.shift) % Lz + Lz) % Lz;
            } else {
                const double zf = op.sgn[2] * d[op.perm[2]] + cz;
                zi = std::lround(zf);
                if (std::fabs(zf - zi) > 1e-9) { ok = false; break; }
            }
            if (std::fabs(xf - xi) > 1e-9 || std::fabs(yf - yi) > 1e-9) { ok = false; break; }
            auto it = index.find({static_cast<int>(xi), static_cast<int>(yi), static_cast<int>(zi)});
            if (it == index.end()) { ok = false; break; }
            img[i] = it->second;
        }
        if (ok) images.push_back(img);
    }
    // an operation that maps every site onto the other sublattice: with it the spin-down lattice
    // Green function is the spin-up one at permuted sites (the lattice step inverts half the
    // matrices)
    for (const auto& im : images) {
        bool all = true;
        for (int i = 0; i < N && all; ++i) all = lat.parity[im[i]] != lat.parity[i];
        if (all) { lat.gdn = im; break; }
    }
    std::vector<int> rep_site(N);
    for (int i = 0; i < N; ++i) {
        int m = i;
        for (auto& im : images) m = std::min(m, im[i]);
        rep_site[i] = m;
    }
    lat.site_rep.assign(N, -1);
    for (int i = 0; i < N; ++i)
        if (rep_site[i] == i) {
            lat.site_rep[i] = static_cast<int>(lat.rep.size());
            lat.rep.push_back(i);
        }
    lat.rep_of.resize(N);
    lat.flip.resize(N);
    for (int i = 0; i < N; ++i) {
        lat.rep_of[i] = lat.site_rep[rep_site[i]];
        lat.flip[i] = lat.parity[i] != lat.parity[rep_site[i]] ? 1 : 0;
    }
    return true;
}

// Bump allocator over the caller's workspace (base == nullptr: size computation only).
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~static_cast<size_t>(255);
        T* ptr = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return ptr;
    }
};

}  // namespace

struct hf_ctx {
    hf_params p{};
    HostLattice lat;
    int L = 0, nsite = 0, nchain = 0, nw = 0;
    double dtau = 0.0, lambda = 0.0;
    double a_p = 0.0, a_m = 0.0, ev_p = 0.0, ev_m = 0.0;
    cudaStream_t stream = nullptr;
    int device = 0;                 // device current at hf_init (the workspace's device)
    int lat_batch = 0;              // matrices per lattice-step launch
    bool lat_wide = false;          // lattice step in the blocked band form
    int wide_npos = 0;              // its listed positions per spin matrix
    std::vector<int> wide_pos_host; // [nspin][wide_npos] host copy of wide_pos
    uint32_t nmeas = 0;             // measured sweeps since the last clear (all chains)
    uint32_t nsw_host = 0;          // sweep counter shared by all chains (FP32 path)
    std::string err;
    // device state
    double* gtau = nullptr;         // [nsite][2][L]
    double* G = nullptr;            // [nchain][2][L*L]
    float* Gf = nullptr;            // [nchain][2][L*L] (precision 1)
    double* g0inv = nullptr;        // [nsite][2][L*L] inverse bath matrices
    bool g0inv_stale = true;        // the baths changed since g0inv was computed
    int8_t* s = nullptr;            // [nchain][L]
    uint32_t* nsw = nullptr;        // [nchain]
    uint32_t* nmeas_d = nullptr;    // [nchain]
    unsigned long long* acc = nullptr;  // [nchain]
    double* bins = nullptr;         // [nchain][max_bins][2L+3]
    int* status = nullptr;          // [8]: [0..3] errors and counters, [4..5] drift monitor
    double* obs_mean = nullptr;     // [nsite][2L+4]
    double* obs_err = nullptr;      // [nsite][2L+4]
    double2* sigma = nullptr;       // [nsite][2][nw]
    double2* gloc = nullptr;
    double2* weiss_inv = nullptr;
    double2* gwt = nullptr;
    double2* gimp = nullptr;
    double2* sigma_new = nullptr;
    double* c23 = nullptr;          // [nsite][2]
    double* h0band = nullptr;       // [N][b+1]
    int* rep_of = nullptr;          // [N]
    int* flip = nullptr;            // [N]
    int* site_rep = nullptr;        // [N]
    int* site_dn = nullptr;         // [N]
    double2* lat_scratch = nullptr; // [lat_batch][N][b+1]
    int* wide_pos = nullptr;        // [nspin][wide_npos] blocked band form: positions to solve for
    int* wide_out = nullptr;        // [nspin][wide_npos] and the gloc row each one fills
    int* lat_work = nullptr;        // [1 + lat_batch] its task counter and ready flags
    // tensor-core refresh of the mixed-precision form (precision 1, L = 128, refresh_gj = 0)
    bool tc_on = false;
    hfk::TcRefreshArgs tc{};
    // phase timing: events on the context stream (see hf_get_timings)
    cudaEvent_t ev[9] = {};
    bool ev_rdmft = false, ev_sweep = false;
    ~hf_ctx() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

hf_status fail(hf_ctx* c, hf_status st, const std::string& msg) {
    if (c) c->err = msg; else g_init_error = msg;
    return st;
}

hf_status cuda_fail(hf_ctx* c, cudaError_t e, const char* what) {
    (void)cudaGetLastError();   // consume it, so that a later launch check does not see it again
    return fail(c, HF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define HF_CUDA(ctx, call)                                             \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
    } while (0)

hf_status validate(const hf_params& p, std::string& err) {
    if (!(p.beta > 0.0) || !(p.dtau > 0.0)) { err = "beta and dtau must be > 0"; return HF_EINVAL; }
    const double Lr = p.beta / p.dtau;
    const int L = static_cast<int>(std::lround(Lr));
    if (std::fabs(Lr - L) > 1e-9 * Lr) { err = "beta / dtau must be an integer"; return HF_EINVAL; }
    if ((p.precision == 0 || p.precision == 2) && !hfk::qmc_f64_supported(L)) {
        err = "FP64 sweeps support L in {8,12,16,20,24,32,40,48,64}, got " + std::to_string(L);
        return HF_EINVAL;
    }
    if (p.precision == 1 && !hfk::qmc_f32_supported(L)) {
        err = "FP32 sweeps support L in {16,32,64,128}, got " + std::to_string(L);
        return HF_EINVAL;
    }
    if (p.precision < 0 || p.precision > 2) { err = "precision must be 0, 1 or 2"; return HF_EINVAL; }
    if (p.chains_per_site < 1) { err = "chains_per_site must be >= 1"; return HF_EINVAL; }
    if (!(p.delay_k == 0 || p.delay_k == 1 || p.delay_k == 4 || p.delay_k == 8 || p.delay_k == 16 ||
          p.delay_k == 32) || (p.delay_k > 1 && p.precision != 2)) {
        err = "delay_k must be 0/1 (rank-1) or, for FP32-pair sweeps (precision 2), 4, 8, 16 or 32";
        return HF_EINVAL;
    }
    if (!(p.team_warps == 0 || p.team_warps == 1 || p.team_warps == 2 || p.team_warps == 4) ||
        (L > 32 && p.team_warps == 1)) {
        err = "team_warps must be 0 (default), 1, 2 or 4, and >= 2 for L > 32";
        return HF_EINVAL;
    }
    if (p.delay_k > 1 && (p.team_warps > 1 || (p.team_warps == 0 && hfk::qmc_default_team_warps(L) > 1))) {
        err = "delay_k > 1 runs with one warp per chain only (team_warps = 1, L <= 32)";
        return HF_EINVAL;
    }
    if (p.precision != 1) {
        const int tw = p.team_warps > 0 ? p.team_warps : hfk::qmc_default_team_warps(L);
        const size_t smem = (p.precision == 2) ? hfk::qmc_df64_smem_bytes(L, tw, p.delay_k)
                                               : hfk::qmc_f64_smem_bytes(L, tw);
        if (smem > static_cast<size_t>(227) * 1024) {
            err = "team_warps / delay_k need " + std::to_string(smem) +
                  " bytes of shared memory per block (limit 232448); use more warps per chain or a "
                  "smaller delay_k";
            return HF_EINVAL;
        }
    }
    if (p.n_matsubara < 1 || p.n_matsubara > 100000) { err = "n_matsubara out of range"; return HF_EINVAL; }
    if (p.bin_size < 1 || p.max_bins < 1) { err = "bin_size and max_bins must be >= 1"; return HF_EINVAL; }
    if (p.refresh_every < 0) { err = "refresh_every must be >= 0"; return HF_EINVAL; }
    if (p.precision == 1 && p.refresh_every < 1) {
        err = "FP32 sweeps need a periodic FP64 refresh (refresh_every >= 1)";
        return HF_EINVAL;
    }
    if (!(p.check_drift == 0 || p.check_drift == 1)) { err = "check_drift must be 0 or 1"; return HF_EINVAL; }
    if (!(p.lattice_form >= 0 && p.lattice_form <= 2)) { err = "lattice_form must be 0, 1 or 2"; return HF_EINVAL; }
    if (!(p.refresh_stagger == 0 || p.refresh_stagger == 1) ||
        (p.refresh_stagger == 1 && p.precision == 1 && p.refresh_every > 1)) {
        err = "refresh_stagger must be 0 or 1; staggered phases need fused refreshes (precision 0 "
              "or 2) unless refresh_every is 1";
        return HF_EINVAL;
    }
    if (p.n_warmup < 0 || p.n_measure < 0) { err = "sweep counts must be >= 0"; return HF_EINVAL; }
    if (!(p.U >= 0.0)) { err = "U must be >= 0"; return HF_EINVAL; }
    if (!(p.mix > 0.0 && p.mix <= 1.0)) { err = "mix must be in (0, 1]"; return HF_EINVAL; }
    if (!std::isfinite(p.t) || !std::isfinite(p.V0) || !std::isfinite(p.mu) || !std::isfinite(p.h_seed)) {
        err = "non-finite model parameter";
        return HF_EINVAL;
    }
    return HF_OK;
}

// Layout of the device state; returns total bytes.  base == nullptr computes sizes only.
size_t layout(hf_ctx& c, void* base) {
    Carver cv(base);
    const int L = c.L, ns = c.nsite, nc = c.nchain, nw = c.nw, N = c.lat.N, bw = c.lat.b + 1;
    c.gtau = cv.take<double>(static_cast<size_t>(ns) * 2 * L);
    c.G = cv.take<double>(static_cast<size_t>(nc) * 2 * L * L);
    c.Gf = c.p.precision == 1 ? cv.take<float>(static_cast<size_t>(nc) * 2 * L * L) : nullptr;
    c.g0inv = cv.take<double>(static_cast<size_t>(ns) * 2 * L * L);
    c.s = cv.take<int8_t>(static_cast<size_t>(nc) * L);
    c.nsw = cv.take<uint32_t>(nc);
    c.nmeas_d = cv.take<uint32_t>(nc);
    c.acc = cv.take<unsigned long long>(nc);
    c.bins = cv.take<double>(static_cast<size_t>(nc) * c.p.max_bins * (2 * L + 3));
    c.status = cv.take<int>(8);
    c.obs_mean = cv.take<double>(static_cast<size_t>(ns) * (2 * L + 4));
    c.obs_err = cv.take<double>(static_cast<size_t>(ns) * (2 * L + 4));
    const size_t nsw2 = static_cast<size_t>(ns) * 2 * nw;
    c.sigma = cv.take<double2>(nsw2);
    c.gloc = cv.take<double2>(nsw2);
    c.weiss_inv = cv.take<double2>(nsw2);
    c.gwt = cv.take<double2>(nsw2);
    c.gimp = cv.take<double2>(nsw2);
    c.sigma_new = cv.take<double2>(nsw2);
    c.c23 = cv.take<double>(static_cast<size_t>(ns) * 2);
    c.h0band = cv.take<double>(static_cast<size_t>(N) * bw);
    c.rep_of = cv.take<int>(N);
    c.flip = cv.take<int>(N);
    c.site_rep = cv.take<int>(N);
    c.site_dn = cv.take<int>(N);
    c.lat_scratch = cv.take<double2>(static_cast<size_t>(c.lat_batch) * N * bw);
    c.wide_pos = cv.take<int>(static_cast<size_t>(4) * ns);
    c.wide_out = cv.take<int>(static_cast<size_t>(4) * ns);
    c.lat_work = cv.take<int>(static_cast<size_t>(c.lat_batch) + 1);
    c.tc_on = c.p.precision == 1 && L == hfk::kTcL && c.p.refresh_gj == 0;
    if (c.tc_on) {
        c.tc.g0inv_digits = cv.take<uint16_t>(hfk::tc_digits_bytes(ns) / 2);
        c.tc.g0inv_rowT = cv.take<int>(static_cast<size_t>(ns) * 2 * L);
        c.tc.scratch = cv.take<double>(static_cast<size_t>(nc) * L * L);
        c.tc.fail = cv.take<int>(nc);
        c.tc.fail_list = cv.take<int>(nc);
        c.tc.fail_count = cv.take<int>(1);
        c.tc.products = cv.take<unsigned long long>(1);
    }
    return cv.off + 256;
}

hf_status setup_sizes(hf_ctx& c, const hf_params* p) {
    if (!p) return fail(nullptr, HF_EINVAL, "null params");
    std::string err;
    hf_status st = validate(*p, err);
    if (st != HF_OK) return fail(nullptr, st, err);
    c.p = *p;
    if (!build_lattice(*p, c.lat, err)) return fail(nullptr, HF_EINVAL, err);
    if (!hfk::lattice_band_supported(c.lat.b))
        return fail(nullptr, HF_EINVAL,
                    "the lattice's band half-width " + std::to_string(c.lat.b) +
                        " exceeds the lattice step's band buffers (largest: " +
                        std::to_string(hfk::lattice_max_band()) + ")");
    // automatic: the window form below the bands whose products run on the tensor cores, the
    // blocked form from there on (and wherever the window does not fit)
    if (p->lattice_form == 2 && !hfk::lattice_window_supported(c.lat.b))
        return fail(nullptr, HF_EINVAL, "lattice_form 2 (the window form) needs a band half-width <= " +
                                             std::to_string(hfk::lattice_window_max_band()));
    c.lat_wide = p->lattice_form == 1 ||
                 (p->lattice_form == 0 && c.lat.b >= hfk::lattice_wide_tc_min_band()) ||
                 !hfk::lattice_window_supported(c.lat.b);
    c.L = static_cast<int>(std::lround(p->beta / p->dtau));
    c.nsite = static_cast<int>(c.lat.rep.size());
    c.nchain = c.nsite * p->chains_per_site;
    c.nw = p->n_matsubara;
    // lattice step: as many (w_n, sigma) matrices per launch as fit in 1 GiB of band buffers
    // (blocked band form: 24 GiB, split evenly over the launches, so that each launch still fills
    // the GPU with one matrix per SM; one launch holds the 500 matrices of the periodic 16^3 box)
    const size_t per = hfk::lattice_scratch_per_matrix(c.lat.N, c.lat.b);
    const int nq = (c.lat.gdn.empty() ? 2 : 1) * c.nw;
    if (c.lat_wide) {
        const size_t cap = std::max<size_t>(1, (static_cast<size_t>(24) << 30) / (per ? per : 1));
        const size_t nl = (static_cast<size_t>(nq) + cap - 1) / cap;
        c.lat_batch = static_cast<int>((static_cast<size_t>(nq) + nl - 1) / nl);
    } else {
        const size_t cap = (static_cast<size_t>(1) << 30) / (per ? per : 1);
        c.lat_batch = static_cast<int>(std::max<size_t>(1, std::min<size_t>(2 * c.nw, cap)));
    }
    return HF_OK;
}

// Multiplier of the sweep kernels' slot-to-chain map: the smallest m > nchain / 4 coprime with
// nchain, so that the chains of one block lie about a quarter of the chain range apart (sites
// across the trap, whose acceptance and hence work differ).  Taken for the FP64 sweeps of one
// context, whose blocks all run in one wave, so that the SMs finish together (measured: square20
// QMC 615 -> 575 ms).  Not for the FP32-pair form, whose blocks gain more from sharing one site's
// g0^{-1} in L1 (216 -> 241 ms with the map), nor for fused batches, which run several waves that
// the block scheduler balances.
int slot_multiplier(int nchain) {
    if (nchain < 8) return 1;
    for (int m = nchain / 4 + 1; m < nchain; ++m) {
        int a = m, b = nchain;
        while (b) { const int t = a % b; a = b; b = t; }
        if (a == 1) return m;
    }
    return 1;
}

hfk::QmcProblem make_problem(const hf_ctx& c, int n_warmup, int n_measure, int refresh_first) {
    hfk::QmcProblem q{};
    q.L = c.L;
    q.cps = c.p.chains_per_site;
    q.nchain = c.nchain;
    q.block0 = 0;
    q.seed_lo = static_cast<uint32_t>(c.p.seed & 0xFFFFFFFFull);
    q.seed_hi = static_cast<uint32_t>(c.p.seed >> 32);
    q.a_p = c.a_p;
    q.a_m = c.a_m;
    q.ev_p = c.ev_p;
    q.ev_m = c.ev_m;
    q.af_p = static_cast<float>(c.a_p);
    q.af_m = static_cast<float>(c.a_m);
    q.afl_p = static_cast<float>(c.a_p - static_cast<double>(q.af_p));
    q.afl_m = static_cast<float>(c.a_m - static_cast<double>(q.af_m));
    q.n_warmup = n_warmup;
    q.n_measure = n_measure;
    q.refresh_every = c.p.refresh_every;
    q.refresh_stagger = c.p.refresh_stagger;
    q.slot_mult = c.p.precision == 0 ? slot_multiplier(c.nchain) : 1;
    q.bin_size = c.p.bin_size;
    q.max_bins = c.p.max_bins;
    q.refresh_first = refresh_first;
    q.team_warps = c.p.team_warps > 0 ? c.p.team_warps : hfk::qmc_default_team_warps(c.L);
    q.delay_k = c.p.delay_k > 1 ? c.p.delay_k : 1;
    q.gtau = c.gtau;
    q.G = c.G;
    q.Gf = c.Gf;
    q.g0inv = c.g0inv;
    q.s = c.s;
    q.nsw = c.nsw;
    q.nmeas = c.nmeas_d;
    q.acc = c.acc;
    q.bins = c.bins;
    q.status = c.status;
    q.drift = c.p.check_drift ? reinterpret_cast<unsigned int*>(c.status + 4) : nullptr;
    return q;
}

hf_status check_status(hf_ctx* c) {
    int st[4] = {0, 0, 0, 0};
    HF_CUDA(c, cudaMemcpyAsync(st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st[0] != 0) {
        HF_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        if (st[0] == HF_EINVAL)   // only the self-checking build reports this
            return fail(c, HF_EINVAL, "device self-check failed at line " + std::to_string(st[2]) +
                                          " (value " + std::to_string(st[3]) + ")");
        return fail(c, static_cast<hf_status>(st[0]),
                    "device reported a numerical failure (singular Dyson matrix or non-finite value)");
    }
    return HF_OK;
}

// g0^{-1} of every site whenever the baths changed since it was last built (stream order).
hf_status ensure_g0inv(hf_ctx* c, cudaStream_t st) {
    if (!c->g0inv_stale) return HF_OK;
    hfk::QmcBatch b{};
    b.nprob = 1;
    b.p[0] = make_problem(*c, 0, 0, 0);
    cudaError_t e = hfk::launch_g0_inverse(b, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "g0 inverse launch");
    if (c->tc_on) {   // the digits of g0^{-1} that the tensor-core refresh multiplies by
        e = hfk::launch_g0inv_digits(b.p[0], c->tc, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "g0 inverse digits launch");
    }
    c->g0inv_stale = false;
    return HF_OK;
}

// Mixed-precision sequence: FP32 sweep segments that end at the chains' next refresh point,
// each followed by the FP64 refresh kernel, which also takes that sweep's measurement (the
// measurement of a refresh sweep comes after the refresh, as in the FP64 path).
hf_status launch_sweeps_f32(hf_ctx* c, int n_warmup, int n_measure, int refresh_first) {
    hfk::QmcProblem q = make_problem(*c, n_warmup, n_measure, refresh_first);
    cudaError_t e = cudaSuccess;
    const hf_status sg = ensure_g0inv(c, c->stream);
    if (sg != HF_OK) return sg;
    if (refresh_first) {
        hfk::QmcProblem q0 = q;
        q0.refresh_measure = 0;
        q0.drift = nullptr;          // the first refresh follows a possible bath change
        e = hfk::launch_refresh_f64(q0, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "FP64 refresh launch");
    }
    const int total = n_warmup + n_measure;
    const uint32_t re = static_cast<uint32_t>(c->p.refresh_every);
    uint32_t nsw = c->nsw_host;
    for (int k = 0; k < total;) {
        const int to_refresh = static_cast<int>(re - (nsw % re));
        const int n = std::min(to_refresh, total - k);
        const bool lands = (n == to_refresh);
        hfk::QmcBatch b{};
        b.nprob = 1;
        b.p[0] = q;
        b.p[0].nsweeps = n;
        b.p[0].meas_from = std::max(0, n_warmup - k);
        b.p[0].meas_to = std::max(b.p[0].meas_from, n - (lands ? 1 : 0));
        b.nblocks = c->nchain;
        e = hfk::launch_qmc_f32(b, hfk::qmc_f32_smem_bytes(c->L), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "FP32 sweep launch");
        if (lands) {
            q.refresh_measure = (k + n - 1 >= n_warmup) ? 1 : 0;
            if (c->tc_on) {
                // Newton steps on the tensor cores from the sweep's FP32 state; a chain whose
                // residual does not converge is refreshed by Gauss-Jordan right after
                e = cudaMemsetAsync(c->tc.fail_count, 0, sizeof(int), c->stream);
                if (e == cudaSuccess) e = hfk::launch_refresh_tc(q, c->tc, c->stream);
                if (e == cudaSuccess)
                    e = hfk::launch_refresh_f64_listed(q, c->tc.fail_list, c->tc.fail_count, c->stream);
            } else {
                e = hfk::launch_refresh_f64(q, c->stream);
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "FP64 refresh launch");
        }
        k += n;
        nsw += static_cast<uint32_t>(n);
    }
    c->nsw_host = nsw;
    return HF_OK;
}

hf_status launch_sweeps(hf_ctx* c, int n_warmup, int n_measure, int refresh_first) {
    if (c->p.precision == 1) return launch_sweeps_f32(c, n_warmup, n_measure, refresh_first);
    const hf_status sg = ensure_g0inv(c, c->stream);
    if (sg != HF_OK) return sg;
    hfk::QmcBatch b{};
    b.nprob = 1;
    b.p[0] = make_problem(*c, n_warmup, n_measure, refresh_first);
    const int tw = b.p[0].team_warps;
    const int cpb = hfk::qmc_f64_chains_per_block(c->L, tw);
    b.nblocks = (c->nchain + cpb - 1) / cpb;
    const size_t smem = (c->p.precision == 2) ? hfk::qmc_df64_smem_bytes(c->L, tw, b.p[0].delay_k)
                                              : hfk::qmc_f64_smem_bytes(c->L, tw);
    cudaError_t e = (c->p.precision == 2) ? hfk::launch_qmc_df64(b, smem, c->stream)
                                          : hfk::launch_qmc_f64(b, smem, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "QMC sweep launch");
    c->nsw_host += static_cast<uint32_t>(n_warmup + n_measure);
    return HF_OK;
}

hfk::LatticeArgs lattice_args(const hf_ctx& c) {
    hfk::LatticeArgs la{};
    la.N = c.lat.N;
    la.b = c.lat.b;
    la.nw = c.nw;
    la.beta = c.p.beta;
    la.mu = c.p.mu;
    la.h0band = c.h0band;
    la.rep_of = c.rep_of;
    la.flip = c.flip;
    la.site_rep = c.site_rep;
    la.site_dn = c.lat.gdn.empty() ? nullptr : c.site_dn;
    la.nspin = c.lat.gdn.empty() ? 2 : 1;
    la.sigma = c.sigma;
    la.gloc = c.gloc;
    la.scratch = c.lat_scratch;
    la.status = c.status;
    la.wide = c.lat_wide ? 1 : 0;
    la.wide_npos = c.wide_npos;
    la.wide_pos = c.wide_pos;
    la.wide_out = c.wide_out;
    la.work = c.lat_work;
    return la;
}

hf_status enqueue_lattice(hf_ctx* c) {
    const hfk::LatticeArgs la = lattice_args(*c);
    const int nq = la.nspin * c->nw;
    for (int q0 = 0; q0 < nq; q0 += c->lat_batch) {
        cudaError_t e = hfk::launch_lattice(la, q0, std::min(c->lat_batch, nq - q0), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "lattice step launch");
    }
    return HF_OK;
}

// Raw generator blocks for hf_philox_blocks: one thread per counter.
__global__ void philox_blocks_kernel(uint2 key, const uint4* __restrict__ ctr, int n,
                                     uint4* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = hfk::philox4x32_10(ctr[k], key);
}

hfk::FourierArgs fourier_args(const hf_ctx& c) {
    hfk::FourierArgs fa{};
    fa.nsite = c.nsite;
    fa.L = c.L;
    fa.nw = c.nw;
    fa.beta = c.p.beta;
    fa.U = c.p.U;
    fa.mix = c.p.mix;
    fa.c23 = c.c23;
    fa.gloc = c.gloc;
    fa.sigma = c.sigma;
    fa.weiss_inv = c.weiss_inv;
    fa.gwt = c.gwt;
    fa.gtau = c.gtau;
    fa.obs_mean = c.obs_mean;
    fa.gimp = c.gimp;
    fa.sigma_new = c.sigma_new;
    return fa;
}

}  // namespace

extern "C" {

hf_status hf_workspace_size(const hf_params* p, size_t* bytes) {
    if (!bytes) return fail(nullptr, HF_EINVAL, "null bytes pointer");
    hf_ctx c;
    hf_status st = setup_sizes(c, p);
    if (st != HF_OK) return st;
    *bytes = layout(c, nullptr);
    return HF_OK;
}

hf_status hf_lattice_info(const hf_params* p, int* N, int* n_sites, int* band, int* spins, int* rep,
                          int* rep_of, int* flip) {
    hf_ctx c;
    hf_status st = setup_sizes(c, p);
    if (st != HF_OK) return st;
    const HostLattice& lat = c.lat;
    if (N) *N = lat.N;
    if (n_sites) *n_sites = static_cast<int>(lat.rep.size());
    if (band) *band = lat.b;
    if (spins) *spins = lat.gdn.empty() ? 2 : 1;
    if (rep) std::memcpy(rep, lat.rep.data(), sizeof(int) * lat.rep.size());
    if (rep_of) std::memcpy(rep_of, lat.rep_of.data(), sizeof(int) * lat.N);
    if (flip) std::memcpy(flip, lat.flip.data(), sizeof(int) * lat.N);
    return HF_OK;
}

hf_status hf_init(const hf_params* p, void* d_ws, size_t ws_bytes, hf_ctx** out) {
    if (!out) return fail(nullptr, HF_EINVAL, "null output handle");
    *out = nullptr;
    hf_ctx* c = new (std::nothrow) hf_ctx();
    if (!c) return fail(nullptr, HF_ENOMEM, "host allocation failed");
    hf_status st = setup_sizes(*c, p);
    if (st != HF_OK) { delete c; return st; }
    const size_t need = layout(*c, nullptr);
    if (!d_ws || ws_bytes < need) {
        delete c;
        return fail(nullptr, HF_ENOMEM, "workspace of " + std::to_string(ws_bytes) +
                                            " bytes is smaller than the " + std::to_string(need) +
                                            " bytes needed");
    }
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255u) != 0) {
        delete c;
        return fail(nullptr, HF_EINVAL, "workspace must be 256-byte aligned");
    }
    layout(*c, d_ws);
    c->stream = static_cast<cudaStream_t>(p->cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return fail(nullptr, HF_ECUDA, "hf_init: no current CUDA device");
    }
    // a1: Trotter step and Hubbard-Stratonovich coupling (host libm)
    c->dtau = p->beta / c->L;
    c->lambda = std::acosh(std::exp(c->dtau * p->U / 2.0));
    c->a_p = std::exp(-2.0 * c->lambda) - 1.0;
    c->a_m = std::exp(2.0 * c->lambda) - 1.0;
    c->ev_p = std::exp(c->lambda) - 1.0;
    c->ev_m = std::exp(-c->lambda) - 1.0;

    const int N = c->lat.N, bw = c->lat.b + 1, ns = c->nsite, nw = c->nw;
    // H0 and the orbit tables in band order (band position k holds site order[k])
    const HostLattice& lat = c->lat;
    std::vector<double> h0(static_cast<size_t>(N) * bw, 0.0);
    std::vector<int> rep_of_k(N), flip_k(N), site_rep_k(N), site_dn_k(N, -1);
    for (int k = 0; k < N; ++k) {
        const int i = lat.order[k];
        h0[static_cast<size_t>(k) * bw] = lat.V[i];
        for (int j : lat.nbr[i])
            if (lat.pos[j] > k) h0[static_cast<size_t>(k) * bw + (lat.pos[j] - k)] += -p->t;
        rep_of_k[k] = lat.rep_of[i];
        flip_k[k] = lat.flip[i];
        site_rep_k[k] = lat.site_rep[i];
    }
    if (!lat.gdn.empty())
        for (int r = 0; r < ns; ++r) site_dn_k[lat.pos[lat.gdn[lat.rep[r]]]] = r;
    // blocked band form: the band position whose G_kk fills each output (r, slot).  In the
    // matrix of spin sp the site at position k carries G of orbit rep_of_k[k] and spin
    // sp ^ flip_k[k], the same at every such site (the symmetries mapping one onto another keep
    // the matrix), so the member with the largest position is taken: its forward solve is the
    // shortest.  Both spins inverted: matrix sp fills slot sp; spin-halved: the spin-up matrix
    // fills both slots, slot 1 from the members on the other sublattice.
    const int nspin = lat.gdn.empty() ? 2 : 1;
    c->wide_npos = ns * (3 - nspin);
    std::vector<int> wpos, wout;
    for (int sp = 0; sp < nspin; ++sp) {
        std::vector<int> best(static_cast<size_t>(ns) * 2, -1);
        for (int k = 0; k < N; ++k) {
            const int slot = sp ^ flip_k[k];
            if (nspin == 2 && slot != sp) continue;
            best[static_cast<size_t>(rep_of_k[k]) * 2 + slot] = k;   // ascending k: the largest wins
        }
        std::vector<std::pair<int, int>> lst;
        for (int r = 0; r < ns; ++r)
            for (int slot = 0; slot < 2; ++slot) {
                if (nspin == 2 && slot != sp) continue;
                const int k = best[static_cast<size_t>(r) * 2 + slot];
                if (k < 0) {
                    delete c;
                    return fail(nullptr, HF_EINVAL, "internal: an orbit has no site for a spin slot");
                }
                lst.emplace_back(k, r * 2 + slot);
            }
        std::sort(lst.begin(), lst.end());
        for (const auto& pr : lst) {
            wpos.push_back(pr.first);
            wout.push_back(pr.second);
        }
    }
    std::vector<double> c23(static_cast<size_t>(ns) * 2);
    std::vector<double2> sig(static_cast<size_t>(ns) * 2 * nw);
    for (int i = 0; i < ns; ++i) {
        const int r = c->lat.rep[i];
        const double c2 = c->lat.V[r] - p->mu + p->U / 2.0;
        c23[2 * i] = c2;
        c23[2 * i + 1] = c2 * c2 + c->lat.z[r] * p->t * p->t;
        for (int sp = 0; sp < 2; ++sp) {
            const double sg = sp == 0 ? 1.0 : -1.0;
            const double v = p->U / 2.0 - sg * p->h_seed * c->lat.parity[r];
            for (int n = 0; n < nw; ++n) sig[(static_cast<size_t>(i) * 2 + sp) * nw + n] = make_double2(v, 0.0);
        }
    }
    cudaStream_t st0 = c->stream;
    auto up = [&](void* dst, const void* src, size_t n) {
        return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st0);
    };
    cudaError_t e = up(c->h0band, h0.data(), h0.size() * sizeof(double));
    if (e == cudaSuccess) e = up(c->rep_of, rep_of_k.data(), N * sizeof(int));
    if (e == cudaSuccess) e = up(c->flip, flip_k.data(), N * sizeof(int));
    if (e == cudaSuccess) e = up(c->site_rep, site_rep_k.data(), N * sizeof(int));
    if (e == cudaSuccess) e = up(c->site_dn, site_dn_k.data(), N * sizeof(int));
    c->wide_pos_host = wpos;
    if (e == cudaSuccess) e = up(c->wide_pos, wpos.data(), wpos.size() * sizeof(int));
    if (e == cudaSuccess) e = up(c->wide_out, wout.data(), wout.size() * sizeof(int));
    if (e == cudaSuccess) e = up(c->c23, c23.data(), c23.size() * sizeof(double));
    if (e == cudaSuccess) e = up(c->sigma, sig.data(), sig.size() * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->gtau, 0, sizeof(double) * ns * 2 * c->L, st0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nsw, 0, sizeof(uint32_t) * c->nchain, st0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nmeas_d, 0, sizeof(uint32_t) * c->nchain, st0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(unsigned long long) * c->nchain, st0);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->bins, 0, sizeof(double) * c->nchain * p->max_bins * (2 * c->L + 3), st0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int) * 8, st0);
    if (e == cudaSuccess && c->tc_on) e = cudaMemsetAsync(c->tc.products, 0, sizeof(unsigned long long), st0);
    if (e == cudaSuccess)
        e = hfk::launch_init_fields(c->s, c->nchain, p->chains_per_site, c->L,
                                    static_cast<uint32_t>(p->seed & 0xFFFFFFFFull),
                                    static_cast<uint32_t>(p->seed >> 32), st0);
    for (int k = 0; k < 9 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev[k]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        std::string m = std::string("hf_init device setup: ") + cudaGetErrorString(e);
        delete c;
        return fail(nullptr, HF_ECUDA, m);
    }
    *out = c;
    return HF_OK;
}

hf_status hf_get_lattice_plan(const hf_ctx* c, int* form, int* launches, double* cfma,
                              double* tc_flops) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    const int N = c->lat.N, b = c->lat.b;
    const int nspin = c->lat.gdn.empty() ? 2 : 1;
    const int nq = nspin * c->nw;
    const int nl = (nq + c->lat_batch - 1) / c->lat_batch;
    double f = 0.0;   // factorisation: d (d + 1) / 2 at column k, d = min(b, N - 1 - k)
    for (int k = 0; k < N; ++k) {
        const double d = std::min(b, N - 1 - k);
        f += d * (d + 1) / 2;
    }
    if (c->lat_wide) {   // forward solves from each listed position p: min(b, N - 1 - j), j >= p
        std::vector<double> tail(static_cast<size_t>(N) + 1, 0.0);
        for (int j = N - 1; j >= 0; --j) tail[j] = tail[j + 1] + std::min(b, N - 1 - j);
        double sv = 0.0;
        for (int p : c->wide_pos_host) sv += tail[p];
        f += sv / nspin;
    } else {             // selected inversion: d^2 + d at column k
        for (int k = 0; k < N; ++k) {
            const double d = std::min(b, N - 1 - k);
            f += d * d + d;
        }
    }
    if (form) *form = c->lat_wide ? 1 : 0;
    if (launches) *launches = nl;
    if (cfma) *cfma = f;
    if (tc_flops)
        *tc_flops = c->lat_wide ? hfk::lattice_wide_tc_flops(N, b, c->wide_pos_host.data(), c->wide_npos, nspin)
                                : 0.0;
    return HF_OK;
}

hf_status hf_get_sizes(const hf_ctx* c, int* n_sites, int* n_chains, int* L, int* N) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (n_sites) *n_sites = c->nsite;
    if (n_chains) *n_chains = c->nchain;
    if (L) *L = c->L;
    if (N) *N = c->lat.N;
    return HF_OK;
}

hf_status hf_get_orbits(const hf_ctx* c, int* rep, int* rep_of, int* flip) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (rep) std::memcpy(rep, c->lat.rep.data(), sizeof(int) * c->nsite);
    if (rep_of) std::memcpy(rep_of, c->lat.rep_of.data(), sizeof(int) * c->lat.N);
    if (flip) std::memcpy(flip, c->lat.flip.data(), sizeof(int) * c->lat.N);
    return HF_OK;
}

hf_status hf_set_g0(hf_ctx* c, int site, int spin, const double* g0_tau) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (site < 0 || site >= c->nsite || spin < 0 || spin > 1 || !g0_tau)
        return fail(c, HF_EINVAL, "hf_set_g0: bad site, spin or pointer");
    for (int m = 0; m < c->L; ++m)
        if (!std::isfinite(g0_tau[m])) return fail(c, HF_EINVAL, "hf_set_g0: non-finite bath value");
    HF_CUDA(c, cudaMemcpyAsync(c->gtau + (static_cast<size_t>(site) * 2 + spin) * c->L, g0_tau,
                               sizeof(double) * c->L, cudaMemcpyHostToDevice, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    c->g0inv_stale = true;
    return HF_OK;
}

hf_status hf_get_g0(hf_ctx* c, double* g0_tau) {
    if (!c || !g0_tau) return fail(c, HF_EINVAL, "hf_get_g0: null argument");
    HF_CUDA(c, cudaMemcpyAsync(g0_tau, c->gtau, sizeof(double) * c->nsite * 2 * c->L,
                               cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_sweep(hf_ctx* c, int n_warmup, int n_measure, int refresh_first) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (n_warmup < 0 || n_measure < 0) return fail(c, HF_EINVAL, "hf_sweep: negative sweep count");
    const uint64_t cap = static_cast<uint64_t>(c->p.max_bins) * c->p.bin_size;
    if (static_cast<uint64_t>(c->nmeas) + n_measure > cap)
        return fail(c, HF_EINVAL, "hf_sweep: measurements would overflow max_bins * bin_size; "
                                  "call hf_clear_measurements first");
    HF_CUDA(c, cudaEventRecord(c->ev[7], c->stream));
    hf_status st = launch_sweeps(c, n_warmup, n_measure, refresh_first);
    if (st != HF_OK) return st;
    HF_CUDA(c, cudaEventRecord(c->ev[8], c->stream));
    c->ev_sweep = true;
    c->nmeas += static_cast<uint32_t>(n_measure);
    return HF_OK;
}

hf_status hf_clear_measurements(hf_ctx* c) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    HF_CUDA(c, cudaMemsetAsync(c->bins, 0, sizeof(double) * c->nchain * c->p.max_bins * (2 * c->L + 3),
                               c->stream));
    HF_CUDA(c, cudaMemsetAsync(c->nmeas_d, 0, sizeof(uint32_t) * c->nchain, c->stream));
    HF_CUDA(c, cudaMemsetAsync(c->status + 4, 0, sizeof(int) * 4, c->stream));
    if (c->tc_on) HF_CUDA(c, cudaMemsetAsync(c->tc.products, 0, sizeof(unsigned long long), c->stream));
    c->nmeas = 0;
    return HF_OK;
}

static hf_status reduce_all(hf_ctx* c) {
    const int nb = static_cast<int>(c->nmeas / c->p.bin_size);
    cudaError_t e = hfk::launch_reduce(c->bins, c->nsite, c->p.chains_per_site, c->L,
                                       c->p.max_bins, nb, c->p.bin_size, c->obs_mean, c->obs_err,
                                       c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduction launch");
    return HF_OK;
}

hf_status hf_measure(hf_ctx* c, int site, double* gtau, double* n, double* d, double* m,
                     double* errs) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (site < 0 || site >= c->nsite) return fail(c, HF_EINVAL, "hf_measure: bad site");
    hf_status st = reduce_all(c);
    if (st != HF_OK) return st;
    const int K = 2 * c->L + 4;
    std::vector<double> mean(K), err(K);
    HF_CUDA(c, cudaMemcpyAsync(mean.data(), c->obs_mean + static_cast<size_t>(site) * K,
                               sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaMemcpyAsync(err.data(), c->obs_err + static_cast<size_t>(site) * K,
                               sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream));
    st = check_status(c);
    if (st != HF_OK) return st;
    const int L = c->L;
    if (gtau) std::memcpy(gtau, mean.data(), sizeof(double) * 2 * L);
    if (n) { n[0] = mean[2 * L]; n[1] = mean[2 * L + 1]; }
    if (d) *d = mean[2 * L + 2];
    if (m) *m = mean[2 * L + 3];
    if (errs) std::memcpy(errs, err.data(), sizeof(double) * K);
    return HF_OK;
}

hf_status hf_get_observables(hf_ctx* c, double* mean, double* err) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    const size_t K = static_cast<size_t>(c->nsite) * (2 * c->L + 4);
    if (mean) HF_CUDA(c, cudaMemcpyAsync(mean, c->obs_mean, sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream));
    if (err) HF_CUDA(c, cudaMemcpyAsync(err, c->obs_err, sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_rdmft_step(hf_ctx* c, double* iter_seconds) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    const uint64_t cap = static_cast<uint64_t>(c->p.max_bins) * c->p.bin_size;
    if (static_cast<uint64_t>(c->p.n_measure) > cap)
        return fail(c, HF_EINVAL, "hf_rdmft_step: n_measure exceeds max_bins * bin_size");
    auto t0 = std::chrono::steady_clock::now();
    HF_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    // a9: lattice step, in chunks of lat_batch (w_n, sigma) matrices
    hf_status st0 = enqueue_lattice(c);
    if (st0 != HF_OK) return st0;
    // Weiss fields and the tau-grid bath
    const hfk::FourierArgs fa = fourier_args(*c);
    HF_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    cudaError_t e = hfk::launch_weiss_tau(fa, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "Weiss-field launch");
    c->g0inv_stale = true;
    HF_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
    // impurities: warm-started chains, fresh bins
    hf_status st = hf_clear_measurements(c);
    if (st != HF_OK) return st;
    HF_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
    st = launch_sweeps(c, c->p.n_warmup, c->p.n_measure, 1);
    if (st != HF_OK) return st;
    HF_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
    c->nmeas = static_cast<uint32_t>(c->p.n_measure);
    st = reduce_all(c);
    if (st != HF_OK) return st;
    HF_CUDA(c, cudaEventRecord(c->ev[5], c->stream));
    e = hfk::launch_sigma_update(fa, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "self-energy update launch");
    HF_CUDA(c, cudaEventRecord(c->ev[6], c->stream));
    c->ev_rdmft = true;
    st = check_status(c);
    if (st != HF_OK) return st;
    auto t1 = std::chrono::steady_clock::now();
    if (iter_seconds) *iter_seconds = std::chrono::duration<double>(t1 - t0).count();
    return HF_OK;
}

hf_status hf_compute_baths(hf_ctx* c) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    hf_status st = enqueue_lattice(c);
    if (st != HF_OK) return st;
    const cudaError_t e = hfk::launch_weiss_tau(fourier_args(*c), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "Weiss-field launch");
    c->g0inv_stale = true;
    return check_status(c);
}

hf_status hf_get_sigma(hf_ctx* c, double* sigma) {
    if (!c || !sigma) return fail(c, HF_EINVAL, "hf_get_sigma: null argument");
    HF_CUDA(c, cudaMemcpyAsync(sigma, c->sigma, sizeof(double2) * c->nsite * 2 * c->nw,
                               cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_set_sigma(hf_ctx* c, const double* sigma) {
    if (!c || !sigma) return fail(c, HF_EINVAL, "hf_set_sigma: null argument");
    HF_CUDA(c, cudaMemcpyAsync(c->sigma, sigma, sizeof(double2) * c->nsite * 2 * c->nw,
                               cudaMemcpyHostToDevice, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_get_gloc(hf_ctx* c, double* gloc) {
    if (!c || !gloc) return fail(c, HF_EINVAL, "hf_get_gloc: null argument");
    HF_CUDA(c, cudaMemcpyAsync(gloc, c->gloc, sizeof(double2) * c->nsite * 2 * c->nw,
                               cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_get_impurity_iw(hf_ctx* c, double* gw0, double* weiss_inv, double* gimp,
                             double* sigma_new) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    const size_t n = sizeof(double2) * c->nsite * 2 * c->nw;
    double* dst[4] = {gw0, weiss_inv, gimp, sigma_new};
    const double2* src[4] = {c->gwt, c->weiss_inv, c->gimp, c->sigma_new};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) HF_CUDA(c, cudaMemcpyAsync(dst[k], src[k], n, cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_get_fields(hf_ctx* c, signed char* fields, uint32_t* counters) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (fields)
        HF_CUDA(c, cudaMemcpyAsync(fields, c->s, static_cast<size_t>(c->nchain) * c->L,
                                   cudaMemcpyDeviceToHost, c->stream));
    if (counters)
        HF_CUDA(c, cudaMemcpyAsync(counters, c->nsw, sizeof(uint32_t) * c->nchain,
                                   cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_set_fields(hf_ctx* c, const signed char* fields, const uint32_t* counters) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (fields) {
        for (size_t i = 0; i < static_cast<size_t>(c->nchain) * c->L; ++i)
            if (fields[i] != 1 && fields[i] != -1)
                return fail(c, HF_EINVAL, "hf_set_fields: fields must be +1 or -1");
        HF_CUDA(c, cudaMemcpyAsync(c->s, fields, static_cast<size_t>(c->nchain) * c->L,
                                   cudaMemcpyHostToDevice, c->stream));
    }
    if (counters) {
        for (int k = 1; k < c->nchain; ++k)
            if (c->p.precision == 1 && counters[k] != counters[0])
                return fail(c, HF_EINVAL, "hf_set_fields: the FP32 path needs equal sweep counters");
        HF_CUDA(c, cudaMemcpyAsync(c->nsw, counters, sizeof(uint32_t) * c->nchain,
                                   cudaMemcpyHostToDevice, c->stream));
        c->nsw_host = counters[0];
    }
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_get_green(hf_ctx* c, int chain, double* G) {
    if (!c || !G) return fail(c, HF_EINVAL, "hf_get_green: null argument");
    if (chain < 0 || chain >= c->nchain) return fail(c, HF_EINVAL, "hf_get_green: bad chain");
    const size_t LL = static_cast<size_t>(c->L) * c->L;
    if (c->p.precision == 0) {
        HF_CUDA(c, cudaMemcpyAsync(G, c->G + static_cast<size_t>(chain) * 2 * LL, sizeof(double) * 2 * LL,
                                   cudaMemcpyDeviceToHost, c->stream));
        HF_CUDA(c, cudaStreamSynchronize(c->stream));
    } else if (c->p.precision == 2) {
        std::vector<float> f(4 * LL);   // (hi, lo) pairs
        HF_CUDA(c, cudaMemcpyAsync(f.data(), c->G + static_cast<size_t>(chain) * 2 * LL,
                                   sizeof(double) * 2 * LL, cudaMemcpyDeviceToHost, c->stream));
        HF_CUDA(c, cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < 2 * LL; ++i)
            G[i] = static_cast<double>(f[2 * i]) + static_cast<double>(f[2 * i + 1]);
    } else {
        std::vector<float> f(2 * LL);
        HF_CUDA(c, cudaMemcpyAsync(f.data(), c->Gf + static_cast<size_t>(chain) * 2 * LL,
                                   sizeof(float) * 2 * LL, cudaMemcpyDeviceToHost, c->stream));
        HF_CUDA(c, cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < 2 * LL; ++i) G[i] = f[i];
    }
    return HF_OK;
}

hf_status hf_get_accepts(hf_ctx* c, unsigned long long* accepts) {
    if (!c || !accepts) return fail(c, HF_EINVAL, "hf_get_accepts: null argument");
    HF_CUDA(c, cudaMemcpyAsync(accepts, c->acc, sizeof(unsigned long long) * c->nchain,
                               cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    return HF_OK;
}

hf_status hf_sync(hf_ctx* c) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    return check_status(c);
}

hf_status hf_get_drift(hf_ctx* c, double* max_drift, unsigned long long* refreshes) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    unsigned int w[2] = {0u, 0u};
    HF_CUDA(c, cudaMemcpyAsync(w, c->status + 4, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    float m = 0.0f;
    std::memcpy(&m, &w[0], sizeof(m));
    if (max_drift) *max_drift = m;
    if (refreshes) *refreshes = w[1];
    return HF_OK;
}

hf_status hf_get_refresh_stats(hf_ctx* c, unsigned long long* tensor_refreshes,
                               unsigned long long* fallbacks, unsigned long long* digit_products) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    unsigned int w[2] = {0u, 0u};
    unsigned long long np = 0ull;
    HF_CUDA(c, cudaMemcpyAsync(w, c->status + 6, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
    if (c->tc_on)
        HF_CUDA(c, cudaMemcpyAsync(&np, c->tc.products, sizeof(np), cudaMemcpyDeviceToHost, c->stream));
    HF_CUDA(c, cudaStreamSynchronize(c->stream));
    if (tensor_refreshes) *tensor_refreshes = w[0];
    if (fallbacks) *fallbacks = w[1];
    if (digit_products) *digit_products = np;
    return HF_OK;
}

hf_status hf_get_timings(hf_ctx* c, double* ms) {
    if (!c || !ms) return fail(c, HF_EINVAL, "hf_get_timings: null argument");
    const int pairs[6][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}, {5, 6}, {7, 8}};
    for (int k = 0; k < 6; ++k) {
        ms[k] = -1.0;
        const bool have = (k < 5) ? c->ev_rdmft : c->ev_sweep;
        if (!have) continue;
        HF_CUDA(c, cudaEventSynchronize(c->ev[pairs[k][1]]));
        float t = 0.0f;
        HF_CUDA(c, cudaEventElapsedTime(&t, c->ev[pairs[k][0]], c->ev[pairs[k][1]]));
        ms[k] = t;
    }
    return HF_OK;
}

hf_status hf_lattice_step_noalloc(hf_ctx* c, const double* d_sigma, double* d_gloc) {
    if (!c) return fail(nullptr, HF_EINVAL, "null context");
    if (!d_sigma || !d_gloc) return fail(c, HF_EINVAL, "hf_lattice_step_noalloc: null pointer");
    const size_t per = hfk::lattice_scratch_per_matrix(c->lat.N, c->lat.b);
    if (per > hfk::lattice_static_scratch_bytes())
        return fail(c, HF_EINVAL,
                    "hf_lattice_step_noalloc: one band of this lattice needs " + std::to_string(per) +
                        " bytes of scratch, more than the " +
                        std::to_string(hfk::lattice_static_scratch_bytes()) +
                        "-byte static array holds; use hf_rdmft_step with a workspace instead");
    int dev = -1;
    HF_CUDA(c, cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(c, HF_EINVAL,
                    "hf_lattice_step_noalloc: the context's device (" + std::to_string(c->device) +
                        ") must be the current device (" + std::to_string(dev) + ")");
    // the same arguments as the lattice phase of hf_rdmft_step, with the caller's buffers and
    // the library's static band array instead of the workspace
    hfk::LatticeArgs la = lattice_args(*c);
    la.sigma = reinterpret_cast<const double2*>(d_sigma);
    la.gloc = reinterpret_cast<double2*>(d_gloc);
    la.scratch = nullptr;
    cudaError_t e = hfk::launch_lattice_static(la, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "hf_lattice_step_noalloc launch");
    return check_status(c);
}

hf_status hf_philox_blocks(uint32_t key_lo, uint32_t key_hi, const uint32_t* d_ctr, int n,
                           uint32_t* d_out, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!d_ctr || !d_out)))
        return fail(nullptr, HF_EINVAL, "hf_philox_blocks: n < 0 or null buffer");
    if (n == 0) return HF_OK;
    if ((reinterpret_cast<uintptr_t>(d_ctr) & 15u) != 0 || (reinterpret_cast<uintptr_t>(d_out) & 15u) != 0)
        return fail(nullptr, HF_EINVAL, "hf_philox_blocks: buffers must be 16-byte aligned");
    philox_blocks_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        make_uint2(key_lo, key_hi), reinterpret_cast<const uint4*>(d_ctr), n,
        reinterpret_cast<uint4*>(d_out));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "hf_philox_blocks launch");
    return HF_OK;
}

hf_status hf_tc_dgemm128(const double* d_A, const double* d_B, double* d_C, int n, int digits,
                         int* d_status, void* cuda_stream) {
    if (n < 0) return fail(nullptr, HF_EINVAL, "hf_tc_dgemm128: n < 0");
    if (digits != 1 && digits != 3 && digits != 5 && digits != 7 && digits != 8)
        return fail(nullptr, HF_EINVAL, "hf_tc_dgemm128: digits must be 1, 3, 5, 7 or 8");
    if (n == 0) return HF_OK;
    if (!d_A || !d_B || !d_C || ((reinterpret_cast<uintptr_t>(d_A) | reinterpret_cast<uintptr_t>(d_B) |
                                   reinterpret_cast<uintptr_t>(d_C)) & 15u) != 0)
        return fail(nullptr, HF_EINVAL, "hf_tc_dgemm128: null or unaligned buffer");
    const cudaError_t e = hfk::launch_tc_dgemm128(d_A, d_B, d_C, n, digits, d_status,
                                                  static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "hf_tc_dgemm128 launch");
    return HF_OK;
}

// ----------------------------------------------------------------------------------------------
// Batches: several contexts (e.g. one RDMFT run per temperature, uneven L) whose impurity sweeps
// run as one fused launch, and whose whole iteration is captured once into a CUDA graph.
// ----------------------------------------------------------------------------------------------
struct hf_batch {
    std::vector<hf_ctx*> ctx;     // in launch order: most expensive chains first
    cudaStream_t stream = nullptr;
    int use_graph = 0;
    int iterations = 0;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
    ~hf_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

static hf_status bfail(hf_batch* b, hf_status st, const std::string& m) {
    if (st == HF_ECUDA) (void)cudaGetLastError();
    if (b) b->err = m; else g_init_error = m;
    return st;
}

// One fused launch of the sweeps of every context in the batch.
static hf_status enqueue_batch_qmc(hf_batch* b, int n_warmup, int n_measure, int refresh_first) {
    hfk::QmcBatch gb{};   // contexts whose baths changed: g0^{-1} first, in one launch
    for (hf_ctx* c : b->ctx)
        if (c->g0inv_stale) gb.p[gb.nprob++] = make_problem(*c, 0, 0, 0);
    if (gb.nprob > 0) {
        const cudaError_t eg = hfk::launch_g0_inverse(gb, b->stream);
        if (eg != cudaSuccess) return bfail(b, HF_ECUDA, std::string("g0 inverse launch: ") + cudaGetErrorString(eg));
        for (hf_ctx* c : b->ctx) c->g0inv_stale = false;
    }
    hfk::QmcBatch qb{};
    qb.nprob = static_cast<int>(b->ctx.size());
    size_t smem = 0;
    int blocks = 0;
    for (int i = 0; i < qb.nprob; ++i) {
        hf_ctx* c = b->ctx[i];
        qb.p[i] = make_problem(*c, n_warmup, n_measure, refresh_first);
        qb.p[i].slot_mult = 1;   // several waves: the block scheduler balances them
        qb.p[i].block0 = blocks;
        const int tw = qb.p[i].team_warps;
        const int cpb = hfk::qmc_f64_chains_per_block(c->L, tw);
        blocks += (c->nchain + cpb - 1) / cpb;
        smem = std::max(smem, c->p.precision == 2 ? hfk::qmc_df64_smem_bytes(c->L, tw, qb.p[i].delay_k)
                                                  : hfk::qmc_f64_smem_bytes(c->L, tw));
    }
    qb.nblocks = blocks;
    const cudaError_t e = (b->ctx[0]->p.precision == 2) ? hfk::launch_qmc_df64(qb, smem, b->stream)
                                                        : hfk::launch_qmc_f64(qb, smem, b->stream);
    if (e != cudaSuccess) return bfail(b, HF_ECUDA, std::string("fused sweep launch: ") + cudaGetErrorString(e));
    return HF_OK;
}

// Every device operation of one batched RDMFT iteration, in stream order (capturable).
static hf_status enqueue_batch_iteration(hf_batch* b) {
    for (hf_ctx* c : b->ctx) {
        hf_status st = enqueue_lattice(c);
        if (st != HF_OK) return bfail(b, st, c->err);
        const cudaError_t e = hfk::launch_weiss_tau(fourier_args(*c), b->stream);
        if (e != cudaSuccess) return bfail(b, HF_ECUDA, "Weiss-field launch");
        c->g0inv_stale = true;
        cudaError_t e1 = cudaMemsetAsync(c->bins, 0, sizeof(double) * c->nchain * c->p.max_bins * (2 * c->L + 3), b->stream);
        cudaError_t e2 = cudaMemsetAsync(c->nmeas_d, 0, sizeof(uint32_t) * c->nchain, b->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess) return bfail(b, HF_ECUDA, "bin clear");
    }
    const int nw = b->ctx[0]->p.n_warmup, nm = b->ctx[0]->p.n_measure;
    hf_status st = enqueue_batch_qmc(b, nw, nm, 1);
    if (st != HF_OK) return st;
    for (hf_ctx* c : b->ctx) {
        const int nb = c->p.n_measure / c->p.bin_size;
        cudaError_t e = hfk::launch_reduce(c->bins, c->nsite, c->p.chains_per_site, c->L, c->p.max_bins, nb,
                                           c->p.bin_size, c->obs_mean, c->obs_err, b->stream);
        if (e == cudaSuccess) e = hfk::launch_sigma_update(fourier_args(*c), b->stream);
        if (e != cudaSuccess) return bfail(b, HF_ECUDA, "reduction / self-energy launch");
    }
    return HF_OK;
}

hf_status hf_batch_create(hf_ctx* const* ctxs, int n, int use_graph, hf_batch** out) {
    if (!out) return bfail(nullptr, HF_EINVAL, "null output handle");
    *out = nullptr;
    if (!ctxs || n < 1 || n > hfk::kMaxProblems)
        return bfail(nullptr, HF_EINVAL, "hf_batch_create: need 1.." + std::to_string(hfk::kMaxProblems) + " contexts");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return bfail(nullptr, HF_EINVAL, "hf_batch_create: null context");
        if (ctxs[i]->stream != ctxs[0]->stream)
            return bfail(nullptr, HF_EINVAL, "hf_batch_create: contexts must share one stream");
        if (ctxs[i]->p.precision == 1 || ctxs[i]->p.precision != ctxs[0]->p.precision)
            return bfail(nullptr, HF_EINVAL, "hf_batch_create: contexts must all use precision 0 or all 2");
        if (ctxs[i]->p.n_warmup != ctxs[0]->p.n_warmup || ctxs[i]->p.n_measure != ctxs[0]->p.n_measure)
            return bfail(nullptr, HF_EINVAL, "hf_batch_create: contexts must share n_warmup and n_measure");
        if (ctxs[i]->p.n_measure > ctxs[i]->p.max_bins * ctxs[i]->p.bin_size)
            return bfail(nullptr, HF_EINVAL, "hf_batch_create: n_measure exceeds max_bins * bin_size");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return bfail(nullptr, HF_EINVAL, "hf_batch_create: repeated context");
    }
    if (use_graph && ctxs[0]->stream == nullptr)
        return bfail(nullptr, HF_EINVAL,
                     "hf_batch_create: graph capture needs the contexts on a created (non-default) stream");
    hf_batch* b = new (std::nothrow) hf_batch();
    if (!b) return bfail(nullptr, HF_ENOMEM, "host allocation failed");
    b->ctx.assign(ctxs, ctxs + n);
    // longest chains first: cost per chain ~ L^3 (sweeps of L proposals, L^2 updates each)
    std::stable_sort(b->ctx.begin(), b->ctx.end(), [](const hf_ctx* a, const hf_ctx* c2) {
        return a->L > c2->L;
    });
    b->stream = ctxs[0]->stream;
    b->use_graph = use_graph;
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
        delete b;
        return bfail(nullptr, HF_ECUDA, "event creation failed");
    }
    *out = b;
    return HF_OK;
}

hf_status hf_batch_sweep(hf_batch* b, int n_warmup, int n_measure, int refresh_first) {
    if (!b) return bfail(nullptr, HF_EINVAL, "null batch");
    if (n_warmup < 0 || n_measure < 0) return bfail(b, HF_EINVAL, "negative sweep count");
    for (hf_ctx* c : b->ctx)
        if (static_cast<uint64_t>(c->nmeas) + n_measure > static_cast<uint64_t>(c->p.max_bins) * c->p.bin_size)
            return bfail(b, HF_EINVAL, "hf_batch_sweep: measurements would overflow max_bins * bin_size");
    if (cudaEventRecord(b->ev0, b->stream) != cudaSuccess) return bfail(b, HF_ECUDA, "event record");
    hf_status st = enqueue_batch_qmc(b, n_warmup, n_measure, refresh_first);
    if (st != HF_OK) return st;
    if (cudaEventRecord(b->ev1, b->stream) != cudaSuccess) return bfail(b, HF_ECUDA, "event record");
    for (hf_ctx* c : b->ctx) {
        c->nmeas += static_cast<uint32_t>(n_measure);
        c->nsw_host += static_cast<uint32_t>(n_warmup + n_measure);
    }
    return HF_OK;
}

hf_status hf_batch_rdmft_step(hf_batch* b, double* gpu_ms) {
    if (!b) return bfail(nullptr, HF_EINVAL, "null batch");
    if (cudaEventRecord(b->ev0, b->stream) != cudaSuccess) return bfail(b, HF_ECUDA, "event record");
    if (!b->use_graph || b->iterations == 0) {
        // first iteration runs uncaptured (it also sets the kernels' launch attributes)
        hf_status st = enqueue_batch_iteration(b);
        if (st != HF_OK) return st;
    } else {
        if (!b->exec) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return bfail(b, HF_ECUDA, "stream capture could not start");
            hf_status st = enqueue_batch_iteration(b);
            const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
            if (st != HF_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (ec != cudaSuccess) return bfail(b, HF_ECUDA, std::string("capture: ") + cudaGetErrorString(ec));
            const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) { b->exec = nullptr; return bfail(b, HF_ECUDA, "graph instantiation failed"); }
        }
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return bfail(b, HF_ECUDA, "graph launch failed");
    }
    if (cudaEventRecord(b->ev1, b->stream) != cudaSuccess) return bfail(b, HF_ECUDA, "event record");
    for (hf_ctx* c : b->ctx) {
        c->nmeas = static_cast<uint32_t>(c->p.n_measure);
        c->nsw_host += static_cast<uint32_t>(c->p.n_warmup + c->p.n_measure);
        hf_status st = check_status(c);
        if (st != HF_OK) return bfail(b, st, c->err);
    }
    ++b->iterations;
    if (gpu_ms) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, b->ev0, b->ev1) != cudaSuccess) return bfail(b, HF_ECUDA, "event timing");
        *gpu_ms = t;
    }
    return HF_OK;
}

hf_status hf_batch_elapsed(hf_batch* b, double* gpu_ms) {
    if (!b || !gpu_ms) return bfail(b, HF_EINVAL, "null argument");
    if (cudaEventSynchronize(b->ev1) != cudaSuccess) return bfail(b, HF_ECUDA, "event sync");
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, b->ev0, b->ev1) != cudaSuccess) return bfail(b, HF_ECUDA, "event timing");
    *gpu_ms = t;
    return HF_OK;
}

void hf_batch_free(hf_batch* b) { delete b; }

const char* hf_batch_last_error(const hf_batch* b) { return b ? b->err.c_str() : g_init_error.c_str(); }

void hf_free(hf_ctx* c) { delete c; }

const char* hf_last_error(const hf_ctx* c) {
    return c ? c->err.c_str() : g_init_error.c_str();
}

}  // extern "C"
