// Batched addition c = a + b (Section 2): map, exclusive carry scan, map.
//
// Work mapping.  The limbs of one instance are cut into chunks of VEC
// consecutive limbs (VEC = 4 when every row is 16-byte aligned, so a chunk is
// one 128-bit load, else 1).  A "team" of lanes holds one instance:
//   * small instances (<= 32 chunks): a team of T = next_pow2(chunks) lanes,
//     several teams per warp; the warp scan is segmented by killing the
//     carry at each team's last lane (the segmented scan of Section 2, with a
//     carry that restarts at every instance);
//   * larger instances: a team of W warps; warp w owns the contiguous chunks
//     [w*R*32, (w+1)*R*32), R rows of 32 chunks, each row one coalesced load.
//     Rows are chained inside the warp, warps through one shared-memory step
//     (the thread -> warp -> block hierarchy of Section 2's footnote).
// Every thread keeps its R chunks in registers (efficient sequentialization,
// Section 2): the limbs are read once and written once, so the kernel is
// bound by HBM bandwidth.
//
// Aligned 256K-bit rows (one team of 8 warps per instance) run a
// persistent, double-buffered form instead: each thread copies its own
// chunks of the CTA's next instance into a private shared-memory stage with
// cp.async while it adds the current one, so a full instance per SM is
// always in flight to HBM whatever the registers allow.
#include "bn_device.cuh"
#include "bn_internal.h"

namespace bn {
namespace {

struct AddArgs {
    const uint32_t *a, *b;
    uint32_t *c;
    uint32_t na, nb, n, nout;
    uint32_t chunks;          // ceil(n / VEC)
    uint32_t team;            // lanes per instance
    uint32_t log2_team;       // sub-warp teams only
    uint32_t kill_mask;       // sub-warp teams: bit set at each team's last lane
    uint32_t warps_per_team;  // multi-warp teams only
    uint32_t teams_per_cta;   // multi-warp teams only
    uint64_t batch;
};

template <int VEC>
__device__ __forceinline__ void load_chunk(const uint32_t *x, uint64_t inst, uint32_t nx, uint32_t j,
                                           bool live, uint32_t (&v)[VEC]) {
    const uint32_t first = j * VEC;
    if (live && first < nx) {
        const uint32_t *p = x + inst * nx + first;
        if constexpr (VEC == 4) {
            uint4 t = ld_stream_v4(p);
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
            v[0] = ld_stream(p);
        }
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[k] = 0;
    }
}

template <int VEC>
__device__ __forceinline__ void store_chunk(uint32_t *row, uint32_t j, const uint32_t (&v)[VEC]) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) st_stream(row + j * VEC + k, v[k]);
}

// Teams of <= 32 lanes: one chunk per lane, segmented warp scan.
template <int VEC>
__global__ void __launch_bounds__(256) k_add_subwarp(AddArgs p) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t inst = gt >> p.log2_team;
    const uint32_t j = (uint32_t)gt & (p.team - 1);
    const bool live = inst < p.batch && j < p.chunks;

    uint32_t a[VEC], b[VEC], s[VEC];
    load_chunk<VEC>(p.a, inst, p.na, j, live, a);
    load_chunk<VEC>(p.b, inst, p.nb, j, live, b);
    const uint32_t g = chunk_add<VEC>(a, b, s);       // step 1: map
    const uint32_t pr = chunk_all_ones<VEC>(s);
    const uint32_t G = __ballot_sync(FULL_MASK, g);    // step 2: segmented scan
    const uint32_t P = __ballot_sync(FULL_MASK, pr);
    const uint64_t X = G & ~p.kill_mask, Y = (G | P) & ~p.kill_mask;
    const uint32_t carries = (uint32_t)(X + Y) ^ (P & ~p.kill_mask);
    const uint32_t cin = (carries >> lane) & 1u;
    if (live) {                                        // step 3: map
        uint32_t *row = p.c + inst * p.nout;
        if (j == p.chunks - 1) st_stream(row + p.n, g | (pr & cin));
        chunk_inc<VEC>(s, cin);
        store_chunk<VEC>(row, j, s);
    }
}

// Teams of W whole warps (W <= 16), R rows of 32 chunks per warp.
constexpr uint32_t kTeamMaxThreads = 512;

// One instance by one team (warp w of the team, team_in_cta within the CTA).
// Every thread of the CTA calls this together (it contains a barrier).
template <int VEC, int R>
__device__ __forceinline__ void add_team_instance(const AddArgs &p, uint64_t inst, bool inst_live,
                                                  uint32_t team_in_cta, uint32_t w, uint32_t *warp_flags) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t j0 = w * R * 32 + lane;

    uint32_t s[R][VEC];
    uint32_t gbits = 0, pbits = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {                      // step 1: map
        const uint32_t j = j0 + r * 32;
        const bool live = inst_live && j < p.chunks;
        uint32_t a[VEC], b[VEC];
        load_chunk<VEC>(p.a, inst, p.na, j, live, a);
        load_chunk<VEC>(p.b, inst, p.nb, j, live, b);
        gbits |= chunk_add<VEC>(a, b, s[r]) << r;
        pbits |= chunk_all_ones<VEC>(s[r]) << r;
    }
    // Row flags are recomputed in step 3 rather than kept: ballots are cheap
    // and R rows of flags would not fit next to R rows of sums.
    uint32_t wg = 0, wp = 1;                           // neutral (no carry, propagate)
#pragma unroll
    for (int r = 0; r < R; ++r) {                      // step 2a: rows, then warp
        const RowFlags f{__ballot_sync(FULL_MASK, (gbits >> r) & 1u),
                         __ballot_sync(FULL_MASK, (pbits >> r) & 1u)};
        uint32_t rg;
        row_carries(f, 0, rg);
        carry_compose(wg, wp, rg, f.P == FULL_MASK);
    }
    if (lane == 0) warp_flags[warp] = wg | (wp << 1);
    __syncthreads();
    // step 2b: scan the team's warp summaries (one lane per warp of the team)
    const uint32_t sw = lane < p.warps_per_team ? warp_flags[team_in_cta * p.warps_per_team + lane] : 0u;
    RowFlags fw{__ballot_sync(FULL_MASK, sw & 1u), __ballot_sync(FULL_MASK, (sw >> 1) & 1u)};
    uint32_t unused;
    uint32_t cin = (row_carries(fw, 0, unused) >> w) & 1u;
    if (!inst_live) return;
    uint32_t *row = p.c + inst * p.nout;
#pragma unroll
    for (int r = 0; r < R; ++r) {                      // step 3: map, row by row
        const RowFlags f{__ballot_sync(FULL_MASK, (gbits >> r) & 1u),
                         __ballot_sync(FULL_MASK, (pbits >> r) & 1u)};
        uint32_t cout;
        const uint32_t ci = (row_carries(f, cin, cout) >> lane) & 1u;
        cin = cout;
        const uint32_t j = j0 + r * 32;
        if (j < p.chunks) {
            if (j == p.chunks - 1)
                st_stream(row + p.n, ((gbits >> r) & 1u) | (((pbits >> r) & 1u) & ci));
            chunk_inc<VEC>(s[r], ci);
            store_chunk<VEC>(row, j, s[r]);
        }
    }
}

// ---- the streaming form ------------------------------------------------------

constexpr uint32_t kStreamThreads = 256;  // one team of 8 warps per CTA

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Instances of exactly chunks = 256 R 16-byte chunks (na = nb = n, aligned
// rows), CTA i taking instances i, i + gridDim.x, ...  Shared memory:
// buf[stage][r][operand][thread], 16 bytes each: thread t only ever reads
// the pieces it copied itself, so cp.async.wait_group (its own copies) is
// the only synchronisation the data needs; the warp flags of the carry scan
// alternate between two sets, so one barrier per instance suffices.
template <int R>
__global__ void __launch_bounds__(kStreamThreads) k_add_stream(AddArgs p) {
    extern __shared__ __align__(16) uint4 buf[];
    __shared__ uint32_t warp_flags[2][kStreamThreads / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t j0 = w * R * 32 + lane;
    auto piece = [&](int stage, int r, int op) -> uint4 * {
        return buf + ((stage * R + r) * 2 + op) * kStreamThreads + tid;
    };
    auto issue = [&](uint64_t inst, int stage) {
        const uint32_t *ar = p.a + inst * p.na, *br = p.b + inst * p.nb;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t j = j0 + r * 32;
            cp_async16(piece(stage, r, 0), ar + 4 * j);
            cp_async16(piece(stage, r, 1), br + 4 * j);
        }
        cp_async_commit();
    };
    int stage = 0;
    uint64_t inst = blockIdx.x;
    if (inst < p.batch) issue(inst, 0);
    for (; inst < p.batch; inst += gridDim.x, stage ^= 1) {
        const uint64_t next = inst + gridDim.x;
        if (next < p.batch) {
            issue(next, stage ^ 1);
            cp_async_wait<1>();  // this instance's pieces are in
        } else {
            cp_async_wait<0>();
        }
        uint32_t s[R][4];
        uint32_t gbits = 0, pbits = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {  // step 1: map
            const uint4 av = *piece(stage, r, 0), bv = *piece(stage, r, 1);
            const uint32_t a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
            gbits |= chunk_add<4>(a, b, s[r]) << r;
            pbits |= chunk_all_ones<4>(s[r]) << r;
        }
        uint32_t wg = 0, wp = 1;  // step 2a: rows, then warp
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const RowFlags f{__ballot_sync(FULL_MASK, (gbits >> r) & 1u), __ballot_sync(FULL_MASK, (pbits >> r) & 1u)};
            uint32_t rg;
            row_carries(f, 0, rg);
            carry_compose(wg, wp, rg, f.P == FULL_MASK);
        }
        if (lane == 0) warp_flags[stage][w] = wg | (wp << 1);
        __syncthreads();
        // step 2b: the 8 warps' summaries
        const uint32_t sw = lane < kStreamThreads / 32 ? warp_flags[stage][lane] : 0u;
        const RowFlags fw{__ballot_sync(FULL_MASK, sw & 1u), __ballot_sync(FULL_MASK, (sw >> 1) & 1u)};
        uint32_t unused;
        uint32_t cin = (row_carries(fw, 0, unused) >> w) & 1u;
        uint32_t *row = p.c + inst * p.nout;
#pragma unroll
        for (int r = 0; r < R; ++r) {  // step 3: map, row by row
            const RowFlags f{__ballot_sync(FULL_MASK, (gbits >> r) & 1u), __ballot_sync(FULL_MASK, (pbits >> r) & 1u)};
            uint32_t cout;
            const uint32_t ci = (row_carries(f, cin, cout) >> lane) & 1u;
            cin = cout;
            const uint32_t j = j0 + r * 32;
            if (j == p.chunks - 1) st_stream(row + p.n, ((gbits >> r) & 1u) | (((pbits >> r) & 1u) & ci));
            chunk_inc<4>(s[r], ci);
            store_chunk<4>(row, j, s[r]);
        }
    }
}

template <int R>
cudaError_t launch_stream(const AddArgs &args, cudaStream_t st) {
    const uint32_t smem = 2u * R * 2u * kStreamThreads * 16u;
    cudaError_t e = allow_max_smem((const void *)k_add_stream<R>);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_add_stream<R>, kStreamThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint64_t ctas = (uint64_t)sms * per_sm;
    const uint32_t grid = (uint32_t)(args.batch < ctas ? args.batch : ctas);
    k_add_stream<R><<<grid, kStreamThreads, smem, st>>>(args);
    return cudaGetLastError();
}

template <int VEC, int R>
__global__ void __launch_bounds__(kTeamMaxThreads) k_add_team(AddArgs p) {
    __shared__ uint32_t warp_flags[kTeamMaxThreads / 32];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t team_in_cta = warp / p.warps_per_team;
    const uint32_t w = warp - team_in_cta * p.warps_per_team;
    const uint64_t inst = (uint64_t)blockIdx.x * p.teams_per_cta + team_in_cta;
    add_team_instance<VEC, R>(p, inst, inst < p.batch, team_in_cta, w, warp_flags);
}

// Mixed-size batch of additions of one size class: team i of the grid takes
// item i (items are sorted largest first); 32-bit loads, any sizes <= the
// class maximum.
template <int R>
__global__ void __launch_bounds__(kTeamMaxThreads)
    k_add_team_batch(const BatchItem *items, uint32_t count, const BatchBinding *bind,
                     uint32_t warps_per_team, uint32_t teams_per_cta) {
    __shared__ uint32_t warp_flags[kTeamMaxThreads / 32];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t team_in_cta = warp / warps_per_team;
    const uint32_t w = warp - team_in_cta * warps_per_team;
    const uint64_t idx = (uint64_t)blockIdx.x * teams_per_cta + team_in_cta;
    const bool live = idx < count;
    BatchItem it{0, 0, 0, 1, 1};
    if (live) it = items[idx];
    AddArgs p{};
    p.a = bind->a + it.off_a;
    p.b = bind->b + it.off_b;
    p.c = bind->c + it.off_c;
    p.na = it.na;
    p.nb = it.nb;
    p.n = it.na > it.nb ? it.na : it.nb;
    p.nout = p.n + 1;
    p.chunks = p.n;
    p.warps_per_team = warps_per_team;
    p.teams_per_cta = teams_per_cta;
    p.batch = 1;
    add_team_instance<1, R>(p, 0, live, team_in_cta, w, warp_flags);
}

uint32_t next_pow2(uint32_t x) {
    uint32_t t = 1;
    while (t < x) t <<= 1;
    return t;
}

uint32_t log2u(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return l;
}

template <int VEC, int R>
cudaError_t launch_team(const AddArgs &args, uint32_t block, uint64_t grid, cudaStream_t st) {
    k_add_team<VEC, R><<<(unsigned)grid, block, 0, st>>>(args);
    return cudaGetLastError();
}

template <int VEC>
cudaError_t launch_team_r(uint32_t R, const AddArgs &args, uint32_t block, uint64_t grid,
                          cudaStream_t st) {
    switch (R) {
    case 1: return launch_team<VEC, 1>(args, block, grid, st);
    case 2: return launch_team<VEC, 2>(args, block, grid, st);
    case 4: return launch_team<VEC, 4>(args, block, grid, st);
    case 8: return launch_team<VEC, 8>(args, block, grid, st);
    }
    if constexpr (VEC == 1) {
        switch (R) {
        case 16: return launch_team<VEC, 16>(args, block, grid, st);
        case 32: return launch_team<VEC, 32>(args, block, grid, st);
        }
    }
    return cudaErrorInvalidConfiguration;
}

constexpr uint32_t kMaxRows4 = 8, kMaxRows1 = 32;

}  // namespace

bn_status add_configure(AddConfig &cfg, uint32_t na, uint32_t nb, const bn_tuning *t) {
    if (na == 0 || nb == 0) return BN_EINVAL;
    if (na > BN_ADD_MAX_LIMBS || nb > BN_ADD_MAX_LIMBS) return BN_EUNSUPPORTED;
    cfg = AddConfig{};
    cfg.na = na;
    cfg.nb = nb;
    cfg.n = na > nb ? na : nb;
    cfg.nout = cfg.n + 1;
    if (t) {
        if (t->reserved || t->variant) return BN_EINVAL;
        if (t->cta_threads && (t->cta_threads % 32 || t->cta_threads > 1024)) return BN_EINVAL;
        uint32_t l = t->limbs_per_thread;
        if (l && (l & (l - 1) || l > 32)) return BN_EINVAL;  // power of two <= 32
        // A team must fit in one CTA for either vector width.
        if (l && (cfg.n + 32 * l - 1) / (32 * l) > kTeamMaxThreads / 32) return BN_EINVAL;
        if (l && l < 4 && (cfg.n + 127) / 128 > kTeamMaxThreads / 32) return BN_EINVAL;
        if (t->cta_threads > kTeamMaxThreads) return BN_EINVAL;
        cfg.limbs_per_thread = l;
        cfg.cta_threads = t->cta_threads;
    }
    return BN_OK;
}

cudaError_t add_launch(const AddConfig &cfg, const uint32_t *a, const uint32_t *b, uint32_t *c,
                       uint64_t batch, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    const bool aligned = (cfg.na % 4 == 0) && (cfg.nb % 4 == 0) &&
                         ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
    const uint32_t vec = aligned ? 4 : 1;
    AddArgs args{};
    args.a = a; args.b = b; args.c = c;
    args.na = cfg.na; args.nb = cfg.nb; args.n = cfg.n; args.nout = cfg.nout;
    args.chunks = (cfg.n + vec - 1) / vec;
    args.batch = batch;

    uint32_t R = 1;
    if (cfg.limbs_per_thread) R = cfg.limbs_per_thread >= vec ? cfg.limbs_per_thread / vec : 1;
    const uint32_t rmax = vec == 4 ? kMaxRows4 : kMaxRows1;
    if (R > rmax) R = rmax;

    if (args.chunks <= 32 && !cfg.limbs_per_thread) {
        args.team = next_pow2(args.chunks);
        args.log2_team = log2u(args.team);
        uint32_t kill = 0;
        for (uint32_t l = args.team - 1; l < 32; l += args.team) kill |= 1u << l;
        args.kill_mask = kill;
        const uint32_t block = cfg.cta_threads ? cfg.cta_threads : 256;
        if (block > 256) return cudaErrorInvalidConfiguration;
        const uint64_t threads = batch << args.log2_team;
        const uint64_t grid = (threads + block - 1) / block;
        if (grid > 0x7fffffffull) return cudaErrorInvalidConfiguration;
        if (vec == 4) k_add_subwarp<4><<<(unsigned)grid, block, 0, st>>>(args);
        else k_add_subwarp<1><<<(unsigned)grid, block, 0, st>>>(args);
        return cudaGetLastError();
    }
    // Multi-warp teams: by default grow the rows per thread until a team has
    // at most 8 warps, then widen the team up to 32 warps.
    uint32_t W = (args.chunks + 32 * R - 1) / (32 * R);
    if (!cfg.limbs_per_thread) {
        while (W > 8 && R < rmax) {
            R *= 2;
            W = (args.chunks + 32 * R - 1) / (32 * R);
        }
    }
    if (W > kTeamMaxThreads / 32) return cudaErrorInvalidConfiguration;
    // Aligned 256K-bit rows (one 8-warp team of 8 rows, registers for two
    // CTAs per SM): the streaming form.  At 64K and 128K bits the team kernel
    // keeps more loads in flight and stays faster (measured on GB300).
    if (vec == 4 && !cfg.limbs_per_thread && !cfg.cta_threads && cfg.na == cfg.nb && W == 8 &&
        R == 8 && args.chunks == 256 * R)
        return launch_stream<8>(args, st);
    args.warps_per_team = W;
    args.team = 32 * W;
    uint32_t target = cfg.cta_threads ? cfg.cta_threads : 256;
    args.teams_per_cta = target > args.team ? target / args.team : 1;
    const uint32_t block = args.team * args.teams_per_cta;
    const uint64_t grid = (batch + args.teams_per_cta - 1) / args.teams_per_cta;
    if (grid > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    return vec == 4 ? launch_team_r<4>(R, args, block, grid, st)
                    : launch_team_r<1>(R, args, block, grid, st);
}

bn_status add_batch_class(AddClass &ac, uint32_t n_max) {
    if (n_max == 0 || n_max > BN_ADD_MAX_LIMBS) return BN_EINVAL;
    ac = AddClass{};
    ac.n_max = n_max;
    uint32_t R = 1, W = (n_max + 31) / 32;
    while (W > 8 && R < kMaxRows1) {
        R *= 2;
        W = (n_max + 32 * R - 1) / (32 * R);
    }
    if (W > kTeamMaxThreads / 32) return BN_EUNSUPPORTED;
    ac.rows = R;
    ac.warps_per_team = W;
    ac.teams_per_cta = 256 > 32 * W ? 256 / (32 * W) : 1;
    ac.block = 32 * W * ac.teams_per_cta;
    return BN_OK;
}

cudaError_t add_batch_launch(const AddClass &ac, const BatchItem *items, uint32_t count,
                             const BatchBinding *bind, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const uint32_t grid = (count + ac.teams_per_cta - 1) / ac.teams_per_cta;
#define BN_ADD_BATCH(RR)                                                                         \
    case RR:                                                                                     \
        k_add_team_batch<RR><<<grid, ac.block, 0, st>>>(items, count, bind, ac.warps_per_team,   \
                                                        ac.teams_per_cta);                       \
        break;
    switch (ac.rows) {
        BN_ADD_BATCH(1) BN_ADD_BATCH(2) BN_ADD_BATCH(4) BN_ADD_BATCH(8) BN_ADD_BATCH(16) BN_ADD_BATCH(32)
    default: return cudaErrorInvalidConfiguration;
    }
#undef BN_ADD_BATCH
    return cudaGetLastError();
}

}  // namespace bn
