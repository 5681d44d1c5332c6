// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include "fgx.h"

namespace fgx {

constexpr int kMaxPasses = 6;
// Workspace header: device status word (offset 0), grid-barrier counter
// (offset 64), phase timeline of 16 globaltimer stamps (offset 128).
constexpr size_t kHeaderBytes = 256;
constexpr int kThreads = 512;
// Largest tile region (tile + ring) of the tiled engine, in elements.
constexpr int kMaxRegion = 1024;

// Geometry of one directional pass over an instance of extents (D, H, W).
// The pass moves along `axis` (0 = D, 1 = H, 2 = W) in direction `dir`; the
// in-line axes are the other two in (D, H, W) order: p (outer) and q (inner).
struct PassGeom {
    int axis, dir;
    int64_t L, P, Q;     // number of lines, in-line extents
    int64_t sl, sp, sq;  // element strides of line, p and q
    int tp, tq;          // tile extents along p and q
    int ntp, ntq;        // tiles along p and q
    int K;               // lines per exchange block (= ring width)
    float t[9];          // (1 - lambda) * |offset|^2 per stencil offset
    float c[9];          // sqrt(t) (the cost itself when lambda = 0)
};

// Edge-cost evaluation modes of the tiled engine (see sweep_kernel.cu);
// kCostFast: the general formula with a fused multiply-add and the
// approximate square root (fgx_options.fast_math).
enum { kCostGeneral = 0, kCostAbs = 1, kCostConst = 2, kCostFast = 3 };

// sqrt.approx.f32 of the fast-math edge cost (one hardware approximation,
// relative error about 2^-22; not the IEEE-rounded root).
__device__ __forceinline__ float fast_sqrt(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct SweepArgs {
    const float* image;  // [nimg][C][N]
    const float* mask;   // [B][N]
    float* dist;         // [B][N]
    int64_t B, C, N;
    int64_t nimg;        // distinct images: instance b reads image b % nimg
    int ndim;
    float v, lambda;
    int iterations, npass;
    PassGeom pass[kMaxPasses];
    uint8_t* codes;               // nullable: [iterations*npass][B][N]
    unsigned long long* flags;    // [B][max_tiles] block-progress tags
    unsigned int* barrier;        // grid barrier counter
    int* status;                  // device status word
    long long timeout_ns;
    int max_tiles;
    int smem_region;              // floats per (D or I-channel) region buffer
    int kmax;                     // most lines per exchange block over the passes
    int cost_mode;                // kCostGeneral / kCostAbs / kCostConst
};

// One tile of one instance for one pass application of the tiled engine.
struct TileJob {
    const float* img;             // instance image [C][N]
    float* dist;                  // instance distance map [N]
    uint8_t* codes;               // this pass application's codes [N] or null
    unsigned long long* flags;    // the instance's tile progress tags
    int64_t N;
    int C, ndim;
    float lambda;
    int seq;                      // increasing pass-application counter (tags)
    int tile;
    int region, kmax;
    int* status;
    long long timeout_ns;
};

// One instance of a batched launch (device-side descriptor).
struct InstDesc {
    const float* image;  // [C][N]
    const float* mask;   // [N]
    float* dist;         // [N]
    int64_t N;
    int C, ndim;
    float v, lambda;
    int napps;           // pass applications: iterations * passes
    int npass;
    int cost_mode;
    int flags_off;       // first progress tag of this instance in the tag array
    int region, kmax;    // this instance's tile buffer geometry
    PassGeom pass[kMaxPasses];
};

// Batched launch: instances advance one pass application per round; within a
// round, each wave assigns whole instances to consecutive thread blocks
// (wave_items[w * grid + block] = instance << 16 | tile, or -1).
struct BatchedArgs {
    const InstDesc* desc;
    int n;
    int rounds;
    const int* round_waves;  // [rounds + 1] first wave of each round
    const int* wave_items;   // [waves][grid]
    unsigned long long* flags;
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
};

// Reverse sweep through recorded parent codes (adjoint_kernel.cu).  Uses the
// same pass geometry and tiling as SweepArgs.
struct AdjointArgs {
    const float* image;      // [B][C][N]
    const uint8_t* codes;    // [iterations*npass][B][N]
    const float* grad_dist;  // [B][N]  dL/dD of the final distance
    float* G[2];             // [B][N]  adjoint ping-pong buffers (workspace)
    float* grad_image;       // [B][C][N] or null
    float* grad_mask;        // [B][N] or null
    int64_t B, C, N;
    int ndim;
    float v, lambda;
    int iterations, npass;
    PassGeom pass[kMaxPasses];
    unsigned long long* flags;
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
    int max_tiles;
    int smem_region;
};

// Host helpers (fgx_api.cu)
// Geometry, tiling and buffer sizes of one instance (B = 1) on the tiled
// engine; fills args (pointers unset) and the device's SM count.
int plan_instance(int ndim, int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                  float lambda, const fgx_options* opt, SweepArgs* args, int* sms);
bool device_pointer(const void* p);
void pass_offsets_t(int ndim, int axis, const float sp[3], float lambda, float t[9]);
void pass_extents(int axis, const int64_t ext[3], PassGeom* g);

// 2D warp-chain forward (chain2d.cu)
size_t chain2d_workspace_bytes(int64_t B, int64_t C, int64_t H, int64_t W,
                               const fgx_options* opt);
int chain2d_geometry(int64_t H, int64_t W, const fgx_options* opt, int* K, int* T, int* tv,
                     int* th);
// 3D forward on register-blocked plane tiles (vol3d.cu): workspace bytes, 0
// when the call does not fit that kernel (the tiled engine runs it instead).
size_t vol3d_workspace_bytes(const SweepArgs& f, const fgx_options* opt, int sms);
bool vol3d_supports(const SweepArgs& f, const fgx_options* opt, int sms);
// resume: start from the distances already in `dist` instead of v * M.
int run_vol3d(const SweepArgs& f, const float* image, const float* mask, float* dist,
              uint8_t* codes, float v, void* workspace, size_t ws_bytes, const fgx_options* opt,
              int sms, void* stream, bool resume = false, int64_t nimg = 0);

// Batched 2D instances on the line-chain kernel (chain2d.cu): the size of
// one instance's argument block, filling it (buffers: exchange words at xb,
// Dw/Dt/Ev/Eh from sec; returns the bytes from sec), the launch geometry and
// the launch (table init of every instance, then the rounds).
size_t chain2d_desc_size();
size_t chain2d_instance_desc(void* desc, const fgx_instance& it, const fgx_options* opt,
                             char* hdr, char* xb, char* sec, size_t* xbytes, int* tiles_v,
                             int* tiles_h);
int chain2d_batched_geometry(int sms, const fgx_options* opt, int* grid, size_t* smem);
int launch_chain2d_batched(const void* desc, int n, int init_channels, int max_wp, int max_hp,
                           int rounds, const int* round_waves, const int* wave_items, int grid,
                           char* hdr, long long timeout_ns, void* stream);

// Batched 3D instances on the plane-tile kernel (vol3d.cu): argument block
// size, filling one (false when the instance does not fit the kernel; with
// desc null only the sizes), launch geometry and the launch (D0, working
// copies and range tests of every instance, the rounds, then the results
// copied out of the pitched working copies).
size_t vol3d_desc_size();
// Arguments of one batched 3D instance (desc null: sizes only).  `work`:
// the instance's working copies (*wbytes bytes: pitched distances and image
// where W is not a multiple of 4, the W passes' transposed copies).
bool vol3d_instance_desc(void* desc, const fgx_instance& it, const SweepArgs& f,
                         const fgx_options* opt, int sms, char* hdr, int* range_flag, char* xb,
                         char* work, size_t* xbytes, size_t* wbytes, int* ci, int* max_tiles,
                         int tiles[kMaxPasses]);
// max_ci: the most staged intensity arrays of an instance (kMaxChannels3 +
// 1 and more: cost tables); tables: the staging ring of single planes.
constexpr int kMaxChannels3 = 3;
int vol3d_batched_geometry(int sms, int max_ci, int tables, const fgx_options* opt, int* grid,
                           size_t* smem);
// `hdr` holds the status word; `barrier` is the launch's grid-barrier
// counter (zero at launch).
int launch_vol3d_batched(const void* desc, int n, int rounds, const int* round_waves,
                         const int* wave_items, int grid, size_t smem, int tables, char* hdr,
                         unsigned int* barrier, long long timeout_ns, int sms, void* stream);

// 2D reverse sweep on warp chains (adj2d.cu).
size_t adj2d_workspace_bytes(int64_t B, int64_t H, int64_t W, int iterations,
                             const fgx_options* opt);
// Optional outputs: g0 (the adjoint of D0, [B][H][W]) and lambda_terms (per
// element terms of dL/dlambda, [B][H][W]).
int run_adj2d(const float* grad_dist, const float* image, const uint8_t* codes,
              float* grad_image, float* grad_mask, int64_t B, int64_t C, int64_t H, int64_t W,
              float v, float lambda, int iterations, void* workspace, size_t ws_bytes,
              const fgx_options* opt, int sms, void* stream, float* g0 = nullptr,
              float* lambda_terms = nullptr);

// 3D reverse sweep on plane tiles (vol3d.cu): workspace bytes (0 when the
// geometry does not fit the kernel) and the run (adjoint kernel, then the
// per-voxel image gradient when grad_image is wanted).
size_t adj3d_workspace_bytes(const SweepArgs& f, int iterations, const fgx_options* opt,
                             int sms);
// Reverse sweep of pass applications [t_lo, t_hi) (t_hi < 0: all of them)
// of a transform of `iterations` iterations; `codes` holds the codes of
// those applications.  in_first: the adjoint of application t_hi - 1 is
// grad_dist (-1) or the workspace's adjoint buffer 0 / 1; *in_next (nullable)
// receives the buffer that holds the adjoint handed to application t_lo - 1.
// clear: zero the gradient accumulators first (the first range of a call).
int run_adj3d(const SweepArgs& f, const float* grad_dist, const float* image,
              const uint8_t* codes, float* grad_image, float* grad_mask, float v, int iterations,
              void* workspace, size_t ws_bytes, const fgx_options* opt, int sms, void* stream,
              float* g0 = nullptr, float* lambda_terms = nullptr, const float* s2 = nullptr,
              int t_lo = 0, int t_hi = -1, int in_first = -1, int* in_next = nullptr,
              bool clear = true);

// Parameter gradients (param_grads.cu): v_terms = mask * g0 per element, then
// grad_lambda / grad_v (device doubles, nullable) = float64 sums of
// lambda_terms / v_terms by a fixed-shape tree.
// float64 partial sums of the parameter gradients (bytes of the scratch)
size_t param_partials_bytes();
int run_param_sums(const float* mask, const float* g0, float* v_terms, const float* lambda_terms,
                   double* grad_lambda, double* grad_v, double* partials, int64_t n, int sms,
                   void* stream);

// Failure-detection check (wait_probe.cu): one bounded wait on a tag that
// nothing writes.
void launch_wait_probe(const unsigned long long* tag, int* status, long long timeout_ns,
                       void* stream);

// Signed transform GDT(M) - GDT(1 - M) (signed.cu): workspace bytes for a
// forward workspace of `forward_bytes` and n elements, and the run.
// Encodes a float32 tiled tensor map (a CUtensorMap of 128 bytes at `map`)
// of rank 1..5: dims innermost first, rows of row_pitch floats (0: dims[0])
// and every higher dimension dense over the lower ones, box extents per
// dimension; NaN fill outside the tensor when nan_fill, else zero.  False
// when the driver's encoder is unavailable or the layout cannot be encoded
// (base not 16-byte aligned, a pitch not a multiple of 16 bytes).
bool encode_map_f32(void* map, const void* base, int rank, const uint64_t* dims,
                    const uint32_t* box, bool nan_fill, uint64_t row_pitch = 0);

// Forward of B transforms of nimg images (B a multiple of nimg; instance b
// reads image b % nimg) with the library's fast kernels; the workspace of
// fgx_geodesic_workspace_size(ndim, B, C, D, H, W).
int run_forward_batch(int ndim, const float* image, int64_t nimg, const float* mask, float* dist,
                      int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                      const float spacing[3], float v, float lambda, int iterations,
                      void* workspace, size_t ws_bytes, const fgx_options* opt, void* stream);

size_t signed_workspace_bytes(size_t forward_bytes, int64_t n);
int run_signed(int ndim, const float* image, const float* mask, float* dist, int64_t B,
               int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3], float v,
               float lambda, int iterations, void* workspace, size_t ws_bytes,
               const fgx_options* opt, void* stream);

int run_chain2d(const float* image, const float* mask, float* dist, uint8_t* codes, int64_t B,
                int64_t C, int64_t H, int64_t W, float v, float lambda, int iterations,
                void* workspace, size_t ws_bytes, const fgx_options* opt, int sms, void* stream,
                int64_t nimg = 0);

// Adjoint launchers (adjoint_kernel.cu)
int launch_adjoint(const AdjointArgs& a, int grid, size_t smem, void* stream);
int adjoint_max_blocks_per_sm(size_t smem, int* blocks);

// Launchers (sweep_kernel.cu)
size_t sweep_smem_bytes(int64_t C, int region, int kmax);
int launch_sweep(const SweepArgs& a, int grid, size_t smem, void* stream);
int launch_batched(const BatchedArgs& a, int grid, size_t smem, void* stream);
int batched_max_blocks_per_sm(size_t smem, int* blocks);
int sweep_max_blocks_per_sm(size_t smem, int* blocks);

}  // namespace fgx
