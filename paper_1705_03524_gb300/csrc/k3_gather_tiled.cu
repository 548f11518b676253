// K3 (tiled), host side: launch shapes (shared-memory ring, tile width,
// resident CTAs), the work items of each job, the bin-group split of single
// launches and the reduction that adds the groups' partial likelihoods. The
// kernels themselves are in k3_tiled_kernels.cuh (see there for the design),
// instantiated per kernel kind in k3_tiled_<kind>.cu.
#include <algorithm>

#include "k3_tiled.h"

namespace swih {
namespace {

constexpr int KMAX = kTiledChainMax;
constexpr int kMaxStages = kTiledMaxStages;
constexpr int kDefaultStages = kTiledDefaultStages;

// map[t][i] = sum over bin groups g (in order) of partial[g][t][i]
__global__ void __launch_bounds__(256)
    gather_reduce_kernel(const float *__restrict__ partial, float *__restrict__ map, int nbg, int nt,
                         int64_t n, int64_t map_stride)
{
    const int64_t total = n * nt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / n, j = i - t * n;
        float v = 0.f;
        for (int g = 0; g < nbg; ++g) v += partial[((int64_t)g * nt + t) * n + j];
        map[t * map_stride + j] = v;
    }
}

}  // namespace

cudaError_t tiled_shape(int kind, int elem_bytes, int gdx, int gdy, int max_w, int B, int nl_per_bin,
                        int n_targets, int want_tx, int want_stages, int want_bb, bool row_map, GatherShape *shape)
{
    const bool gau = kind == kGatherGaussian;
    const int A = 16 / elem_bytes;
    const int per_bin = gau ? 2 * gdx + 1 : nl_per_bin;
    const int want = want_stages > 0 ? std::min(want_stages, kMaxStages) : kDefaultStages;
    // wide tiles amortise the window halo; narrow ones when wide segments do
    // not fit, and by default for the register-heavy Gaussian (more resident
    // CTAs per SM)
    int txs[2] = {256, 128};
    int ntx = 2;
    if (want_tx == 128 || (want_tx == 0 && gau)) {
        txs[0] = 128;
        ntx = 1;
    } else if (want_tx == 256) {
        ntx = 1;
    }
    for (int i = 0; i < ntx; ++i) {
        const int tx = txs[i];
        // bins per pipeline step (4 by default). Steps of 2 bins exist for the
        // 256-column 32-bit kernels only, on request (they keep 4 Euclidean CTAs
        // resident, which measured slower than 4-bin steps)
        int bb = gau ? 1 : (want_bb == 8 ? 8 : 4);
        if (!gau && tx == 256 && elem_bytes == 4 && want_bb == 2) bb = 2;
        GatherShape sh;
        sh.tx = tx;
        sh.bb = bb;
        sh.seg = (tx + max_w + 2 * A + A - 1) / A * A;
        sh.nl = bb * per_bin;
        sh.kchain_max = gau ? KMAX : KMAX / 2;
        sh.n_targets = std::max(1, std::min(n_targets, kMaxTargets));
        // shared memory: barriers | sqrt(targets) | likelihood sums | bin-block list | [Gaussian carry] | stages
        // (+ the CTA's list of bin blocks and of their rows to load: 2 x (B + 1) ints, and, when
        // rows are read through a row map, each bin's stored row per lattice row: B x kTiledRowSlots int16)
        sh.dtop_off = (16 * kMaxStages + 4 * sh.n_targets * B + 4 * sh.n_targets * sh.kchain_max * tx + 8 * (B + 1) +
                       (row_map ? 2 * B * kTiledRowSlots : 0) + 15) / 16 * 16;
        const int carry = gau ? (2 * gdx + 1) * (2 * gdy + 1) * tx * 8 : 0;
        sh.stage_off = (sh.dtop_off + carry + 127) / 128 * 128;
        const size_t stage = (size_t)sh.nl * sh.seg * elem_bytes;
        // stages: enough to cover the copy latency, few enough that the CTAs
        // the register file allows stay resident
        TiledOp rq;
        rq.what = TiledOp::kRegs;
        tiled_dispatch(kind, elem_bytes, gdx, gdy, tx, bb, rq);
        const int regs = std::max(rq.regs, 16);
        int ctas = std::min(2048 / (tx + 32), 65536 / ((tx + 32) * ((regs + 7) / 8 * 8)));
        ctas = std::max(ctas, 1);
        // the Gaussian's long steps want at least three stages (one consumed,
        // two in flight) more than one more resident CTA; the cheap kernels
        // want resident CTAs. Settle for two stages when nothing deeper fits.
        // the 256-column 32-bit Manhattan/Euclidean table kernel keeps a copy of
        // its job's parameters past the layout
        const size_t extra = ((kind == kGatherManhattan || kind == kGatherEuclidean) && tx == 256 &&
                              (bb == 4 || bb == 2) && elem_bytes == 4)
                                 ? sizeof(GatherParams)
                                 : 0;
        int ns = 0;
        for (int min_ns = std::min(gau ? 3 : 2, want); min_ns >= 2 && ns < 2; --min_ns) {
            for (int c = ctas; c >= 1; --c) {
                const size_t budget = (size_t)227 * 1024 / c - 1024 - extra;
                if (budget < sh.stage_off + (size_t)min_ns * stage) continue;
                ns = (int)std::min<size_t>(want, (budget - sh.stage_off) / stage);
                break;
            }
        }
        if (ns < 2) continue;
        sh.nstage = ns;
        sh.smem = sh.stage_off + ns * stage;
        sh.ctas_per_sm = std::max(1, std::min(ctas, (int)((size_t)227 * 1024 / (sh.smem + extra + 1024))));
        *shape = sh;
        return cudaSuccess;
    }
    return cudaErrorNotSupported;
}

int tiled_items(GatherParams *job, const GatherShape &shape)
{
    const int h = 2 * job->ry + 1;
    const int slots = (job->ncy + h - 1) / h;
    const int kmax = shape.kchain_max;
    const int nb = std::max(1, (slots + kmax - 1) / kmax);
    job->kchain = (slots + nb - 1) / nb;
    job->nblk = nb;
    job->seg = shape.seg;
    job->nl = shape.nl;
    job->nstage = shape.nstage;
    job->stage_off = shape.stage_off;
    job->dtop_off = shape.dtop_off;
    if (job->nbg < 1) job->nbg = 1;
    if (job->ncx <= 0 || job->ncy <= 0) return 0;
    const int tiles = (job->ncx + shape.tx - 1) / shape.tx;
    return tiles * h * nb * job->nbg;
}

namespace {

// Bin groups for one launch: the count (1, 2, 4 or 8) that minimises the
// modelled time, (waves of resident CTAs) x (bin blocks per CTA + c), with c
// one bin block of fixed cost per CTA (pipeline fill, set-up, output), so a
// launch of 1.6 waves is split into many short CTAs rather than leaving its
// second wave 40% empty.
int choose_bin_groups(const GatherParams &p, const GatherShape &sh, long long base_ctas)
{
    if (!p.map || !p.partial || p.partial_cap <= 0) return 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long res = (long long)std::max(1, sms) * sh.ctas_per_sm;
    const int nbb = (p.B + sh.bb - 1) / sh.bb;
    const double c = 1.0;
    int best = 1;
    double best_cost = (double)((base_ctas + res - 1) / res) * (nbb + c);
    for (int g = 2; g <= 8 && g <= nbb; g *= 2) {
        if ((long long)g * p.n_targets * p.ncx * p.ncy > p.partial_cap) break;
        const int per = (nbb + g - 1) / g;
        if ((g - 1) * per >= nbb) continue;  // a group without bins would leave its partials unwritten
        const double cost = (double)((base_ctas * g + res - 1) / res) * (per + c);
        if (cost < 0.85 * best_cost) {  // CTA times vary, so the model overstates small gains
            best = g;
            best_cost = cost;
        }
    }
    return best;
}

}  // namespace

cudaError_t launch_gather_tiled(const GatherParams &p_in, int kind, int elem_bytes, cudaStream_t s)
{
    if (kind == kGatherWedding) return cudaErrorNotSupported;  // nested windows: the direct gather
    if (p_in.H > kTiledMaxRows) return cudaErrorNotSupported;  // rows beyond int16: the direct gather
    if (p_in.ncx <= 0 || p_in.ncy <= 0) return cudaSuccess;
    GatherShape sh;
    cudaError_t e = tiled_shape(kind, elem_bytes, p_in.gdx, p_in.gdy, 2 * p_in.rx + 1, p_in.B, p_in.nl,
                                p_in.n_targets, p_in.want_tx, p_in.want_stages, p_in.want_bb, true, &sh);
    if (e != cudaSuccess) return e;
    GatherParams p = p_in;
    p.nbg = 1;
    const long long base = tiled_items(&p, sh);
    p.nbg = choose_bin_groups(p, sh, base);
    if ((long long)(2 * p.ry + 1) * p.nblk * p.nbg > 65535) p.nbg = 1;
    if ((long long)(2 * p.ry + 1) * p.nblk > 65535) return cudaErrorNotSupported;
    TiledOp op;
    op.what = TiledOp::kSingle;
    op.p = &p;
    op.sh = &sh;
    op.s = s;
    e = tiled_dispatch(kind, elem_bytes, p.gdx, p.gdy, sh.tx, sh.bb, op);
    if (e != cudaSuccess || p.nbg == 1) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n = (int64_t)p.ncx * p.ncy;
    const long long blocks = std::min<long long>((n * p.n_targets + 255) / 256, (long long)std::max(1, sms) * 8);
    count_launches(1);
    gather_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(p.partial, p.map, p.nbg, p.n_targets, n,
                                                          p.n_targets > 1 ? p.map_stride : 0);
    return cudaGetLastError();
}

cudaError_t launch_gather_table(const GatherParams *d_jobs, const int *d_item_start, int n_jobs,
                                int n_items, const GatherParams &shape_job, int kind, int elem_bytes,
                                int gdx, int gdy, const GatherShape &shape, cudaStream_t s)
{
    (void)shape_job;
    if (n_items <= 0) return cudaSuccess;
    TiledOp op;
    op.what = TiledOp::kTable;
    op.sh = &shape;
    op.d_jobs = d_jobs;
    op.d_items = d_item_start;
    op.n_jobs = n_jobs;
    op.n_items = n_items;
    op.s = s;
    return tiled_dispatch(kind, elem_bytes, gdx, gdy, shape.tx, shape.bb, op);
}

}  // namespace swih
