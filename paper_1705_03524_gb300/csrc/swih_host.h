// Host-side internals shared by the C-ABI translation units: the plan object,
// layout and job-parameter construction, and the work set that lays out and
// launches many regions and window jobs at once (batches, the server).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "swih.h"
#include "swih_internal.h"

struct swih_plan_s {
    swih_plan_desc desc;
    int elem_bytes = 4;
    int n_terms = 0;
    int term_p[swih::kMaxPlanTerms];
    int term_q[swih::kMaxPlanTerms];
    int term_index[swih::kMaxP][swih::kMaxQ];  // [p][q] -> term or -1
    // scan chains: distinct q values and their p lists
    int n_q = 0;
    int q_val[swih::kMaxQ];
    int p_count[swih::kMaxQ];
    int p_val[swih::kMaxQ][swih::kMaxP];
    int gauss_degree = 2;
    double sigma_frac = 0.25;
    int64_t bins_pitch = 0, ih_pitch = 0, plane = 0;
    int band_rows = 0, n_bands = 0;
    int scan_E = 4, scan_threads = 32;
    uint64_t off_ih = 0, off_agg = 0, off_incl = 0, off_flags = 0, total = 0;
    uint64_t flags_bytes = 0;
    uint64_t off_partial = 0, partial_floats = 0;  // split-gather scratch
    // sparse rows (bands of at most 64 rows): rows without a pixel of a bin are
    // not stored; occ holds each (bin, band)'s stored-row mask, row_map each
    // (bin, row)'s last stored row
    bool sparse_rows = false;
    uint64_t off_occ = 0, off_row_map = 0;
    uint64_t off_jobs = 0;  // job tables of swih_likelihood_scales: kJobSlots slots of
                            // SWIH_MAX_SCALES jobs + item starts
    // host copies of the slots' contents and their last use: a call whose table
    // equals a slot's reuses it without an upload
    static constexpr int kJobSlots = 8;
    std::vector<unsigned char> job_slot[kJobSlots];
    uint64_t job_slot_use[kJobSlots] = {};
    uint64_t job_clock = 0;
    // exponential kernel: decay per pixel, fixed-point fraction bits, the four
    // directional integral histograms and the scan's band carries
    bool has_exp = false;
    double exp_lambda = 0.1;
    int exp_F = 0;
    int exp_E = 8, exp_threads = 32;  // exponential scan: columns per thread, threads per block
    uint64_t off_exp = 0, off_exp_carry = 0, off_exp_rows = 0;
    char *d_mem = nullptr;
    uint32_t *d_status = nullptr;
    int device = 0;
    bool built = false;
    int inject = 0;  // SWIH_INJECT_* for the next swih_build_ih
    int gather_path = 0;  // 0: tiled when it fits, 1: direct gather only
    int cfg_tx[5] = {0, 0, 0, 0, 0};      // tiled gather tile width per kernel (0: automatic)
    int cfg_stages[5] = {0, 0, 0, 0, 0};  // tiled gather ring depth per kernel (0: automatic)
    int cfg_bb[5] = {0, 0, 0, 0, 0};      // tiled gather bins per step per kernel (0: automatic)
    // feature channels (swih_plan_channels): n_ch bin planes of H x bins_pitch
    // at offset 0; channel c owns the global bins [ch_bin0[c], ch_bin0[c + 1])
    int n_ch = 0;  // 0: a plan over one image (swih_plan)
    swih_channel_desc ch[SWIH_MAX_CHANNELS];
    int ch_bin0[SWIH_MAX_CHANNELS + 1] = {};
    uint64_t off_chtgt = 0;  // per-channel target table [n_ch][bins] (floats)
    std::string err;
};

namespace swih {

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
inline bool odd_window(int w) { return w >= 3 && (w & 1); }

// per-thread detail string behind swih_last_error(NULL)
std::string &thread_error();
// record msg on the plan (or the thread when plan is NULL) and return st
swih_status fail(swih_plan_s *plan, swih_status st, const std::string &msg);
swih_status cuda_fail(swih_plan_s *plan, const char *what, cudaError_t e);
// total weight of an integer-valued kernel over a w x h window
long double int_kernel_mass(int kernel, int w, int h);
// validate a plan description and fill the plan's term set, ring and layout
swih_status build_layout(const swih_plan_desc *d, swih_plan_s *pl);
// gather parameters of one kernel and window over the plan's integral histograms
swih_status make_gather(swih_plan_s *pl, int kernel, int w, int h, GatherParams &g, int &kind);
// the Gaussian at a w x h window takes the any-degree gather (degree above 2
// or the 128-bit ring), and its parameters
bool gauss_is_wide(const swih_plan_s *pl, int w, int h);
swih_status make_gauss_wide(swih_plan_s *pl, int w, int h, GaussWideParams &g);
// allocate a laid-out plan's workspace on the current device and hand it out
// (the plan is deleted on failure)
swih_status allocate_plan(swih_plan_s *pl, swih_plan_t *out);
// after quantisation into the plan's bin planes: K2, the row map and K2e
swih_status build_scans(swih_plan_s *pl, cudaStream_t s);
// a kernel and window the built plan serves
swih_status check_window(swih_plan_s *pl, int kernel, int w, int h);
// the tiled gather when its row segments fit in shared memory, else the direct one
cudaError_t run_gather(swih_plan_s *pl, const GatherParams &g, int kind, cudaStream_t s);
// floor(exp(-lambda n) 2^64): the fixed-point power q^n of the exponential kernel (n >= 1)
unsigned long long exp_pow_fixed(long double lambda, long double n);

// ---------------------------------------------------------------- work sets
// Settings shared by every region of a work set.
struct WorkSpec {
    int pixel_type = SWIH_PIXEL_U8;
    int bitdepth = 8;
    int bins = 16;
    uint32_t kernel_mask = 0;
    int gauss_degree = 0;
    double gauss_sigma_frac = 0.0;
    int precision = SWIH_PREC_AUTO;
    int band_rows = 0;
    // the term set and ring must also serve windows up to this size (0: only
    // the jobs' windows); lets a set without jobs build integral histograms a
    // later set's jobs read
    int want_win_w = 0, want_win_h = 0;
};

// An image rectangle whose integral histograms are built: H x W pixels at
// image (device), rows pitch bytes apart.
struct WorkRegion {
    const void *image = nullptr;
    int64_t pitch = 0;
    int H = 0, W = 0;
    // Prebuilt (pre_ih != NULL): the region's integral histograms already exist
    // (built by another work set with the same term set, ring and bins); the set
    // neither quantises nor scans it and its jobs read them there. image is then
    // unused. pre_row_map: its row map, or NULL when every row is stored.
    const void *pre_ih = nullptr;
    const int *pre_row_map = nullptr;
    int64_t pre_ih_pitch = 0, pre_plane = 0;
};

// Likelihood maps of one kernel and window over a rectangle of centres of a
// region (region coordinates; the whole valid rectangle when ncx = ncy = 0),
// for n_targets target histograms (target t at target + t * target_stride)
// scored against the same window histograms. Map t is ncy x ncx floats at
// map + t * map_stride.
struct WorkJob {
    int region = 0;
    int kernel = 0;
    int w = 3, h = 3;
    int cx0 = 0, cy0 = 0, ncx = 0, ncy = 0;
    const float *target = nullptr;
    float *map = nullptr;
    int n_targets = 1;
    int64_t target_stride = 0, map_stride = 0;
};

// Lays out the bins, integral histograms, scan state, region and job tables
// and a status word of a set of regions and jobs in one block of device
// memory, and enqueues the three table-driven launches (K1 over every region,
// K2 over every region, K3 once per group of jobs with the same kernel and
// fitted degrees). One term set and one ring serve every region: those a
// plan for the largest region and the largest window would use.
class WorkSet {
  public:
    // host only: validate and lay out; bytes() is then the memory it needs
    swih_status plan(const WorkSpec &spec, const std::vector<WorkRegion> &regions,
                     const std::vector<WorkJob> &jobs, std::string &err);
    uint64_t bytes() const { return total_; }
    // place in device memory (bytes() bytes, 256-byte aligned) and build the
    // host image of the tables (device pointers included)
    swih_status bind(char *d_mem, std::string &err);
    // the tables' host image and their place in device memory
    const void *tables() const { return blob_.data(); }
    size_t tables_bytes() const { return blob_.size(); }
    char *tables_device() const { return d_mem_ + off_tables_; }
    uint32_t *status_device() const { return reinterpret_cast<uint32_t *>(d_mem_ + off_status_); }
    // clear the scan state (and the status block when zero_status), then K1, K2, K3.
    // ev (optional, 1 + n_groups() events): ev[0] is recorded after the scan and
    // row map, ev[1 + g] after job group g's gathers.
    cudaError_t enqueue(cudaStream_t s, bool zero_status, cudaEvent_t const *ev = nullptr) const;
    // integral-histogram bytes the tiled gathers requested, one 64-bit counter
    // per GatherKind (0..4), in the status block (cleared with it)
    unsigned long long *load_counters_device() const
    {
        return reinterpret_cast<unsigned long long *>(d_mem_ + off_status_) + 1;
    }
    // autotuning: per job group
    int n_groups() const { return (int)groups_.size(); }
    bool group_tiled(int g) const { return groups_[g].tiled; }
    int group_kind(int g) const { return groups_[g].kind; }
    void set_group_want(int g, int tx, int stages, int bb);
    void group_want(int g, int &tx, int &stages, int &bb) const;
    swih_status rebuild(std::string &err);  // jobs and tables again, after set_group_want
    cudaError_t enqueue_group(int g, cudaStream_t s) const;
    uint64_t n_evaluations() const { return n_centres_; }  // (centre, window, target) triples
    int elem_bytes() const { return tmpl_.elem_bytes; }
    int n_terms() const { return tmpl_.n_terms; }
    // term set and ring as one comparable value: sets whose signatures are equal
    // can read each other's integral histograms (prebuilt regions)
    std::string signature() const;
    // where region i's integral histograms live (after bind)
    WorkRegion region_as_prebuilt(int i) const;
    int n_built() const { return (int)built_.size(); }

  private:
    struct Region {
        WorkRegion in;
        bool prebuilt = false;
        int n_bands = 0;
        int64_t bins_pitch = 0, ih_pitch = 0, plane = 0;
        uint64_t off_bins = 0, off_ih = 0, off_agg = 0, off_incl = 0, off_flags = 0;
        uint64_t off_occ = 0, off_row_map = 0;  // sparse rows
        int ticket0 = 0;
        long long chunk0 = 0;
    };
    struct Group {
        int kind = 0, gdx = 0, gdy = 0;
        int job_begin = 0, job_end = 0;
        bool tiled = true;
        GatherShape shape{};
        int n_items = 0;
        int items_off = 0;
        int want_tx = 0, want_stages = 0, want_bb = 0;
    };
    swih_status build_jobs(std::string &err);
    void build_blob();

    WorkSpec spec_;
    swih_plan_s tmpl_;
    std::vector<Region> regions_;
    std::vector<int> built_;  // regions this set quantises and scans, in ticket order
    std::vector<WorkJob> in_jobs_;
    std::vector<GatherParams> jobs_;
    std::vector<int> items_;
    std::vector<Group> groups_;
    std::vector<unsigned char> blob_;
    int scan_E_ = 4, scan_threads_ = 32, band_rows_ = 32;
    bool sparse_ = false;  // the scan stores only the rows that hold each bin; gathers read through row maps
    long long scan_tiles_ = 0, quant_chunks_ = 0;
    uint64_t flags_ints_ = 0, n_centres_ = 0;
    uint64_t off_status_ = 0, off_flags_ = 0, off_tables_ = 0, total_ = 0;
    uint64_t tab_quant_ = 0, tab_scan_ = 0, tab_jobs_ = 0, tab_items_ = 0;  // within the tables
    char *d_mem_ = nullptr;
};

}  // namespace swih
