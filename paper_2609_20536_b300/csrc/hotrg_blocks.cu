// Charge-block planning for the block-sparse contractions.
//
// With U(1) (or Z2) symmetry the tensor obeys a charge rule: T[l,r,u,d] is
// zero unless q_l + q_u = q_r + q_d (mod 2 for Z2), and the projector
// P[a,b,x] is zero unless q_x = q_a + q_b (the fused charge of its sector,
// §2.3.1).  Every contraction of a step, written as C = A B^T with row index
// set M, contraction set K and column index set N, is then block diagonal:
// each element of M, K and N carries a value v (a signed sum of its legs'
// labels) and A[m, k] B[n, k] can be nonzero only when v(m) = v(k) = v(n).
// The planner sorts each index set by v (a deterministic counting sort: one
// warp per 256-element chunk, ranks from warp vote masks, no atomics on the
// order), and lays out one group per value present in both M and N:
//   rows of the group  -> positions mbase .. mbase + M_g - 1 of the sorted M list
//   padded slice rows  -> mpad .. mpad + round_up(M_g, 128) - 1
//   tiles              -> tile_base .. + ceil(M_g/128) ceil(N_g/tile_n) - 1 (tile_n = 128 or 64).
// For every position it stores the two element offsets the engine needs
// (operand and output for M and N, A and B for K), and for an output in a pair
// layout a third (the row's or column's part of the pair table index).  Groups whose value has
// no element of K still get tiles: their block of C is zero and is written.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "internal.cuh"

namespace hotrg {

// Value and the three offsets of element idx (sets have < 2^31 elements and
// extents < 2^16, so the mixed-radix decode runs in 32-bit arithmetic).
__device__ __forceinline__ int bs_value(const BsSet& S, int sym, int64_t idx64, int64_t& o0, int64_t& o1,
                                        int64_t& o2) {
    int v = 0;
    o0 = 0;
    o1 = 0;
    o2 = 0;
    uint32_t idx = (uint32_t)idx64;
    for (int f = S.nf - 1; f >= 0; --f) {
        const uint32_t e = (uint32_t)S.f[f].ext;
        const uint32_t q = idx / e;
        const uint32_t i = idx - q * e;
        idx = q;
        v += S.f[f].sgn * S.f[f].lab[i];
        o0 += (int64_t)i * S.f[f].st0;
        o1 += (int64_t)i * S.f[f].st1;
        o2 += (int64_t)i * S.f[f].st2;
    }
    if (sym == SYM_Z2) v &= 1;
    if (sym == SYM_NONE) v = 0;
    return v;
}

constexpr int BS_WARPS = 8;  // warps per block in the counting passes

// Table centre of one product: value v goes to slot v - centre + BS_VOFF.
// The centre stays 0 while every value the legs allow lies in
// [-BS_VOFF, BS_V - BS_VOFF); otherwise it is the midpoint of that range.  In
// the ordered phase the kept U(1) window can drift away from charge 0 (an
// exact +-q pair split at the cut keeps +q, and the fused charge q_a + q_b
// doubles an off-centre window every two steps) while its span stays small,
// so a centred table still holds it.  One block: warp w takes leg w % 3 of
// set w / 3 (its min and max label); thread 0 adds up the signed ranges.
__global__ void __launch_bounds__(32 * 9) bs_centre_kernel(BsSet M, BsSet K, BsSet N, int sym,
                                                            int32_t* __restrict__ centre,
                                                            int32_t* __restrict__ totals) {
    __shared__ int lmin[9], lmax[9];
    for (int i = threadIdx.x; i < 3 * BS_V; i += blockDim.x) totals[i] = 0;  // the count pass adds into them
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const BsSet& S = w < 3 ? M : (w < 6 ? K : N);
    const int f = w % 3;
    int lo = INT_MAX, hi = INT_MIN;
    if (f < S.nf)
        for (int64_t i = lane; i < S.f[f].ext; i += 32) {
            const int q = S.f[f].lab[i];
            lo = min(lo, q);
            hi = max(hi, q);
        }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        lmin[w] = lo;
        lmax[w] = hi;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (sym != SYM_U1) {
        *centre = 0;
        return;
    }
    int64_t vlo = INT64_MAX, vhi = INT64_MIN;
    for (int s = 0; s < 3; ++s) {
        const BsSet& T = s == 0 ? M : (s == 1 ? K : N);
        int64_t a = 0, b = 0;
        for (int g = 0; g < T.nf; ++g) {
            const int64_t mn = lmin[s * 3 + g], mx = lmax[s * 3 + g];
            if (mn > mx) continue;  // a leg without labels contributes nothing
            a += T.f[g].sgn > 0 ? mn * T.f[g].sgn : mx * T.f[g].sgn;
            b += T.f[g].sgn > 0 ? mx * T.f[g].sgn : mn * T.f[g].sgn;
        }
        vlo = a < vlo ? a : vlo;
        vhi = b > vhi ? b : vhi;
    }
    if (vlo >= -BS_VOFF && vhi < BS_V - BS_VOFF) {
        *centre = 0;
    } else {
        const int64_t c = vlo + (vhi - vlo) / 2;
        *centre = (int32_t)(c > INT32_MAX / 2 ? INT32_MAX / 2 : (c < INT32_MIN / 2 ? INT32_MIN / 2 : c));
    }
}

// The three index sets (M, K, N) of a product go through one launch of each
// counting pass: blockIdx.y selects the set.
struct BsSets3 {
    BsSet S[3];
    int32_t* tab[3];  // counts (count pass) or chunk starts (place pass), value-major
    int64_t nch[3];
    int64_t* off0[3];
    int64_t* off1[3];
    int32_t* off2[3];  // null: the set has no pair-table part
    int32_t* totals;   // [3][BS_V] elements per value (count pass)
};

// counts[value][chunk]: elements of each value in every BS_CHUNK-element chunk (value-major,
// so that the single-block scan reads each value's counts contiguously).
__global__ void __launch_bounds__(32 * BS_WARPS) bs_count_kernel(BsSets3 sets, int sym,
                                                                 const int32_t* __restrict__ centre, int32_t* status) {
    __shared__ int32_t tab[BS_WARPS][BS_V];
    const BsSet& S = sets.S[blockIdx.y];
    int32_t* __restrict__ counts = sets.tab[blockIdx.y];
    const int64_t nchunks = sets.nch[blockIdx.y];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int shift = BS_VOFF - *centre;
    const int64_t chunk = (int64_t)blockIdx.x * BS_WARPS + w;
    for (int v = lane; v < BS_V; v += 32) tab[w][v] = 0;
    __syncwarp();
    if (chunk >= nchunks) return;
    const int64_t lo = chunk * BS_CHUNK, hi = min(lo + BS_CHUNK, S.size);
    for (int64_t b = lo; b < hi; b += 32) {
        const int64_t idx = b + lane;
        const bool act = idx < hi;
        int64_t o0, o1, o2;
        const int v = act ? bs_value(S, sym, idx, o0, o1, o2) + shift : -1;
        // an element whose value falls outside the table is left out here and in the
        // placing pass alike (so every counted position is written) and fails the run
        const bool ok = act && v >= 0 && v < BS_V;
        if (act && !ok) atomicExch(status, (int)HOTRG_ENOTSUP);
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
        const unsigned m = __match_any_sync(0xffffffffu, ok ? v : -1) & okm;
        if (ok && (__ffs(m) - 1) == lane) tab[w][v] += __popc(m);
        __syncwarp();
    }
    for (int v = lane; v < BS_V; v += 32) {
        const int32_t c = tab[w][v];
        counts[(int64_t)v * nchunks + chunk] = c;
        if (c) atomicAdd(&sets.totals[blockIdx.y * BS_V + v], c);  // integer sums: any order gives the same
    }
}

// One block of 1024 threads (32 warps): per-value bases from the count pass's
// totals, per-chunk starts of every value present (a warp per value: a
// warp-wide exclusive scan over the chunks, 128 at a time), the group table.
// Values absent from a set need no starts: the placing pass never reads them.
constexpr int BS_SCAN_THREADS = 1024;

__global__ void __launch_bounds__(BS_SCAN_THREADS) bs_scan_kernel(const int32_t* __restrict__ cM, int64_t nM,
                                                       const int32_t* __restrict__ cK, int64_t nK,
                                                       const int32_t* __restrict__ cN, int64_t nN,
                                                       const int32_t* __restrict__ totals,
                                                       int32_t* __restrict__ sM, int32_t* __restrict__ sK,
                                                       int32_t* __restrict__ sN, BsGroup* __restrict__ groups,
                                                       BsHeader* __restrict__ hdr, double* prof_acc, int prof_class,
                                                       int kp_cap, int tile_n, int32_t* status) {
    __shared__ int64_t tot[3][BS_V], base[3][BS_V];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int v = threadIdx.x;  // thread 0 below builds the group table
    const int32_t* cs[3] = {cM, cK, cN};
    int32_t* ss[3] = {sM, sK, sN};
    const int64_t ns[3] = {nM, nK, nN};
    for (int i = threadIdx.x; i < 3 * BS_V; i += blockDim.x) tot[i / BS_V][i % BS_V] = totals[i];
    __syncthreads();
    if (v == 0)
        for (int s = 0; s < 3; ++s) {
            int64_t run = 0;
            for (int u = 0; u < BS_V; ++u) {
                base[s][u] = run;
                run += tot[s][u];
            }
        }
    __syncthreads();
    for (int s = 0; s < 3; ++s)
        for (int u = warp; u < BS_V; u += nw) {
            if (tot[s][u] == 0) continue;
            int64_t run = base[s][u];
            const int32_t* cu = cs[s] + (int64_t)u * ns[s];
            int32_t* su = ss[s] + (int64_t)u * ns[s];
            for (int64_t c0 = 0; c0 < ns[s]; c0 += 128) {
                int32_t x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {  // four loads in flight
                    const int64_t c = c0 + 32 * q + lane;
                    x[q] = c < ns[s] ? cu[c] : 0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int32_t inc = x[q];  // inclusive scan over 32 chunks
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    const int64_t c = c0 + 32 * q + lane;
                    if (c < ns[s]) su[c] = (int32_t)(run + inc - x[q]);
                    run += __shfl_sync(0xffffffffu, inc, 31);
                }
            }
        }
    if (v == 0) {
        int G = 0;
        int64_t mpad = 0, npad = 0, tiles = 0;
        double fl = 0.0, opnd = 0.0, outp = 0.0;
        for (int u = 0; u < BS_V; ++u) {
            if (tot[0][u] == 0 || tot[2][u] == 0) continue;
            BsGroup g;
            g.mbase = base[0][u];
            g.kbase = base[1][u];
            g.nbase = base[2][u];
            g.M = (int32_t)tot[0][u];
            g.K = (int32_t)tot[1][u];
            g.N = (int32_t)tot[2][u];
            g.Kp = (g.K + 31) / 32 * 32;
            if (g.Kp > kp_cap) {  // the slice pitch is too small for this block: fail the run, touch nothing
                atomicExch(status, (int)HOTRG_ENOTSUP);
                g.Kp = 0;
                g.K = 0;
            }
            g.mpad = mpad;
            g.npad = npad;
            g.tiles_n = (g.N + tile_n - 1) / tile_n;
            g.tile_base = (int32_t)tiles;
            mpad += (g.M + 127) / 128 * 128;
            npad += (g.N + 127) / 128 * 128;
            tiles += (int64_t)((g.M + 127) / 128) * g.tiles_n;
            fl += 2.0 * (double)g.M * (double)g.N * (double)g.K;
            opnd += ((double)g.M + (double)g.N) * (double)g.K;
            outp += (double)g.M * (double)g.N;
            groups[G++] = g;
        }
        hdr->G = G;
        hdr->total_tiles = (int32_t)tiles;
        hdr->mpad_total = mpad;
        hdr->npad_total = npad;
        hdr->flops = fl;
        if (prof_acc) {
            prof_acc[prof_class] += fl;
            prof_acc[3 + prof_class] += opnd;
            prof_acc[6 + prof_class] += outp;
        }
    }
}

// Writes the offsets of every element at its sorted position (blockIdx.y = set).
__global__ void __launch_bounds__(32 * BS_WARPS) bs_place_kernel(BsSets3 sets, int sym,
                                                                 const int32_t* __restrict__ centre) {
    __shared__ int32_t tab[BS_WARPS][BS_V];
    const BsSet& S = sets.S[blockIdx.y];
    const int32_t* __restrict__ starts = sets.tab[blockIdx.y];
    const int64_t nchunks = sets.nch[blockIdx.y];
    int64_t* __restrict__ off0 = sets.off0[blockIdx.y];
    int64_t* __restrict__ off1 = sets.off1[blockIdx.y];
    int32_t* __restrict__ off2 = sets.off2[blockIdx.y];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t chunk = (int64_t)blockIdx.x * BS_WARPS + w;
    if (chunk >= nchunks) return;
    const int shift = BS_VOFF - *centre;
    for (int v = lane; v < BS_V; v += 32) tab[w][v] = starts[(int64_t)v * nchunks + chunk];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t lo = chunk * BS_CHUNK, hi = min(lo + BS_CHUNK, S.size);
    for (int64_t b = lo; b < hi; b += 32) {
        const int64_t idx = b + lane;
        const bool act = idx < hi;
        int64_t o0 = 0, o1 = 0, o2 = 0;
        int v = act ? bs_value(S, sym, idx, o0, o1, o2) + shift : -1;
        const bool ok = act && v >= 0 && v < BS_V;
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
        const unsigned m = __match_any_sync(0xffffffffu, ok ? v : -1) & okm;
        int32_t pos = 0;
        if (ok) pos = tab[w][v] + __popc(m & lt);
        __syncwarp();
        if (ok && (__ffs(m) - 1) == lane) tab[w][v] += __popc(m);
        __syncwarp();
        if (ok) {
            off0[pos] = S.pi0 ? (int64_t)S.pi0[o0] : o0;
            off1[pos] = o1;
            if (off2) off2[pos] = (int32_t)o2;
        }
    }
}

static int64_t a256(int64_t x) { return (x + 255) & ~(int64_t)255; }

size_t bs_plan_bytes(int64_t nM, int64_t nK, int64_t nN) {
    size_t b = 0;
    for (int64_t n : {nM, nK, nN}) {
        const int64_t ch = (n + BS_CHUNK - 1) / BS_CHUNK;
        b += 2 * a256(ch * BS_V * 4) + 2 * a256(n * 8) + a256(n * 4);
    }
    b += a256(3 * BS_V * 4);  // per-value totals
    return b + a256(sizeof(BsGroup) * BS_V) + a256(sizeof(BsHeader)) + 256;
}

hotrg_status bs_plan(hotrg_ctx* ctx, int sym, const BsSet& M, const BsSet& K, const BsSet& N, int prof_class,
                     BsPlan& out, int32_t kp_cap_override, int tile_n, const int32_t* pi_out) {
    if (tile_n != 64 && tile_n != 128) return set_err(ctx, HOTRG_EINVAL, "tile width must be 64 or 128");
    const BsSet* sets[3] = {&M, &K, &N};
    int32_t* counts[3];
    int32_t* starts[3];
    int64_t* offs[3][2];
    int32_t* offs2[3] = {nullptr, nullptr, nullptr};
    int64_t nch[3];
    for (int s = 0; s < 3; ++s) {
        nch[s] = (sets[s]->size + BS_CHUNK - 1) / BS_CHUNK;
        counts[s] = (int32_t*)ws_alloc(ctx, nch[s] * BS_V * 4);
        starts[s] = (int32_t*)ws_alloc(ctx, nch[s] * BS_V * 4);
        offs[s][0] = (int64_t*)ws_alloc(ctx, sets[s]->size * 8);
        offs[s][1] = (int64_t*)ws_alloc(ctx, sets[s]->size * 8);
        if (!counts[s] || !starts[s] || !offs[s][0] || !offs[s][1])
            return set_err(ctx, HOTRG_ENOMEM, "block plan workspace exhausted");
        // the output's pair-table parts: rows (M) and columns (N)
        if (pi_out && s != 1 && !(offs2[s] = (int32_t*)ws_alloc(ctx, sets[s]->size * 4)))
            return set_err(ctx, HOTRG_ENOMEM, "block plan workspace exhausted");
    }
    out.groups = (BsGroup*)ws_alloc(ctx, sizeof(BsGroup) * BS_V);
    out.hdr = (BsHeader*)ws_alloc(ctx, sizeof(BsHeader));
    int32_t* centre = (int32_t*)ws_alloc(ctx, 256);
    int32_t* totals = (int32_t*)ws_alloc(ctx, 3 * BS_V * 4);
    if (!out.groups || !out.hdr || !centre || !totals)
        return set_err(ctx, HOTRG_ENOMEM, "block plan workspace exhausted");
    int32_t* st = umma_status_word(ctx);
    if (!st) return set_err(ctx, HOTRG_ENOMEM, "status word");
    cudaStream_t s = ctx->stream;
    bs_centre_kernel<<<1, 32 * 9, 0, s>>>(M, K, N, sym, centre, totals);
    BsSets3 t3;
    t3.totals = totals;
    int64_t nch_max = 1;
    for (int i = 0; i < 3; ++i) {
        t3.S[i] = *sets[i];
        t3.tab[i] = counts[i];
        t3.nch[i] = nch[i];
        t3.off0[i] = offs[i][0];
        t3.off1[i] = offs[i][1];
        t3.off2[i] = offs2[i];
        nch_max = std::max(nch_max, nch[i]);
    }
    const dim3 grid3((unsigned)((nch_max + BS_WARPS - 1) / BS_WARPS), 3);
    bs_count_kernel<<<grid3, 32 * BS_WARPS, 0, s>>>(t3, sym, centre, st);
    double* facc = (ctx->prof.on && ctx->prof.dflops && prof_class >= 0 && prof_class < 3) ? ctx->prof.dflops : nullptr;
    // slice pitch: the whole K set for small sets and Z2 (two blocks); half of it for larger U(1)
    // sets, whose blocks hold a small fraction of K (the device checks every block against it)
    out.kp_cap = kp_cap_override > 0 ? kp_cap_override : bs_pitch(K.size, sym);
    bs_scan_kernel<<<1, BS_SCAN_THREADS, 0, s>>>(counts[0], nch[0], counts[1], nch[1], counts[2], nch[2], totals,
                                      starts[0], starts[1],
                                      starts[2], out.groups, out.hdr, facc, prof_class, out.kp_cap, tile_n, st);
    for (int i = 0; i < 3; ++i) t3.tab[i] = starts[i];
    bs_place_kernel<<<grid3, 32 * BS_WARPS, 0, s>>>(t3, sym, centre);
    HOTRG_COUNT(4);
    HOTRG_LAUNCH_CHECK(ctx, "block planner");
    out.offM0 = offs[0][0];
    out.offM1 = offs[0][1];
    out.offK0 = offs[1][0];
    out.offK1 = offs[1][1];
    out.offN0 = offs[2][0];
    out.offN1 = offs[2][1];
    out.pi_out = pi_out;
    out.kA_contig = K.pi0 != nullptr ? 1 : 0;
    out.offM2 = offs2[0];
    out.offN2 = offs2[2];
    out.tile_n = tile_n;
    out.nM = M.size;
    out.nK = K.size;
    out.nN = N.size;
    return HOTRG_OK;
}

// Pair table (see pair_table): one warp per pair, its lanes counting the pairs that come
// before it; the legs' labels are staged in shared memory.
constexpr int PT_WARPS = 8, PT_MAX = 1024;  // legs of up to PT_MAX indices

__device__ __forceinline__ int pair_value(int qa, int qb, int sym) {
    return sym == SYM_Z2 ? ((qa + qb) & 1) : (sym == SYM_NONE ? 0 : qa + qb);
}

__global__ void __launch_bounds__(32 * PT_WARPS) pair_table_kernel(const int32_t* __restrict__ qa, int na,
                                                                   const int32_t* __restrict__ qb, int nb,
                                                                   int sym, int32_t* __restrict__ pi) {
    __shared__ int32_t sa[PT_MAX], sb[PT_MAX];
    for (int t = threadIdx.x; t < na; t += blockDim.x) sa[t] = qa[t];
    for (int t = threadIdx.x; t < nb; t += blockDim.x) sb[t] = qb[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = na * nb;
    for (int e = blockIdx.x * PT_WARPS + w; e < n; e += gridDim.x * PT_WARPS) {
        const int a = e / nb, b = e - a * nb;
        const int v = pair_value(sa[a], sb[b], sym);
        int cnt = 0;
        for (int a2 = 0; a2 < na; ++a2) {
            const int q = sa[a2];
            for (int b2 = lane; b2 < nb; b2 += 32) {
                const int v2 = pair_value(q, sb[b2], sym);
                cnt += (v2 < v || (v2 == v && a2 * nb + b2 < e)) ? 1 : 0;
            }
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) pi[e] = cnt;
    }
}

hotrg_status pair_table(hotrg_ctx* ctx, int sym, const int32_t* qa, int na, const int32_t* qb, int nb, int32_t* pi) {
    if (na < 1 || nb < 1 || na > PT_MAX || nb > PT_MAX)
        return set_err(ctx, HOTRG_EINVAL, "pair table legs must have 1..1024 indices");
    const int64_t n = (int64_t)na * nb;
    const int blocks = (int)std::min<int64_t>((n + PT_WARPS - 1) / PT_WARPS, (int64_t)ctx->sm_count * 8);
    pair_table_kernel<<<blocks, 32 * PT_WARPS, 0, ctx->stream>>>(qa, na, qb, nb, sym, pi);
    HOTRG_COUNT(1);
    HOTRG_LAUNCH_CHECK(ctx, "pair_table_kernel");
    return HOTRG_OK;
}

}  // namespace hotrg
