// kernels.h -- host-side launchers of the device kernels (one translation unit each
// for the FP32 mover, the FP64 mover, the field phase, the sort and the I/O kernels).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace bitpic {

struct MoveArgs;

// ---- mover (mover_f32.cu, mover_f64.cu) ---------------------------------------
// `move` = false deposits the loaded particles without moving them (the density
// phase of the initial field); `sub`: some species is subcycled; `mixed`: magnetized and
// unmagnetized instances in one batch; `sort`: the step also sorts the store by cell
// into the other copy (MoveArgs.cursor, .d*); `lean` (FP32, a plain step of a batch
// without magnetic field): the variant that queues collision-clock tests for the event
// kernel instead of drawing them inline; `gridv`: the inline-test partner of the mover
// pair, which runs only on the steps where every clock tests (without subcycling: the
// variant that draws a quad's four tests side by side); `kept`: the neutral particle
// targets (whose deposit is kept from step to step) move on this step (on the other
// steps their tiles are skipped).  Returns the launch error.
cudaError_t launch_move_f32(const MoveArgs& a, bool mag, bool move, bool sub, bool mixed,
                            bool sort, bool lean, bool gridv, bool kept, int nt, int grid,
                            cudaStream_t st);
cudaError_t launch_move_f64(const MoveArgs& a, bool mag, bool move, bool sub, bool mixed,
                            bool sort, bool kept, int nt, int grid, cudaStream_t st);
// The rare events the mover queued this step (events.cu): collision candidates, clock
// tests and wall hits, one thread each, `grid` blocks of 128 threads.
cudaError_t launch_events(const MoveArgs& a, int precision, int grid, cudaStream_t st);
// Ionizations against neutral particle targets: convert the requested targets into
// ions (events.cu); one warp per target cell on the step's request list.
cudaError_t launch_victims(const MoveArgs& a, int precision, int grid, cudaStream_t st);
// The y drift of 2-D species after the mover (MoveArgs.yp non-null), before the events.
cudaError_t launch_drift_y(const MoveArgs& a, int precision, int grid, cudaStream_t st);
// resident blocks per SM of the mover variant (0 on error)
// subtest: the grid of a batch whose plain steps run the variant with subcycling and the
// inline clock test (a subcycled colliding species, or a batch below the mover pair's size);
// gridv: the grid of the pair's inline-test partner without subcycling
int move_blocks_per_sm_f32(bool mag, bool sort, bool yp, bool subtest, bool gridv, int nt);
int move_blocks_per_sm_f64(bool mag, bool sort, bool yp, int nt);

// ---- field phase and bookkeeping (field.cu) -------------------------------------
struct FieldArgs {
    const SegParams* seg;
    const InstParams* inst;
    int ninst;
    int max_nodes;                    // max ncells+1 over instances
    unsigned long long* dep;          // accumulating deposit (zeroed by emit)
    unsigned long long* dep_last;     // copy of the last complete deposit
    void* accel;                      // T pairs (A_j, A_{j+1} - A_j), node arrays per segment
    int64_t seg_nodes;                // entries of the segment node arrays (all segments)
    int precision;                    // PIC_FP32 / PIC_FP64
    double* E;                        // per instance node arrays
    // chunks of kChunk nodes: instance of each chunk, and per chunk the partial
    // sums of the interior charge and of the weighted charge, and its first node's charge
    const int* chunk_inst;
    int nchunks;
    i128* part_sum;
    i128* part_w;
    i128* zfirst;
    int64_t* step;                    // [0] the step; an advancing emit sets [1] = [0] + 1
    i128* zs;                         // per instance node arrays: 4x the smoothed node
                                      // charge (instances with the smoother), else unused
    int any_poisson;
};
cudaError_t launch_field(const FieldArgs& f, bool advance_step, cudaStream_t st);
// potential of instance `inst` (FIELD_POISSON) into phi[0..N]
cudaError_t launch_potential(const FieldArgs& f, int inst, double dx, double* phi,
                             cudaStream_t st);

// Snapshot each segment's slot count, rounded up to a whole quad, as the count to
// move, and build the tile prefix (tiles of `tile_quads` quads).
// Also empties the rare-event queue and the target request list of the coming step
// (rare_count[0] and [1]) and sets the step its kernels read: step[0] = step[1].
cudaError_t launch_tiles(const SegParams* seg, unsigned long long* seg_n, int64_t* seg_nmove,
                         int64_t* tile_start, int nseg, int tile_quads,
                         unsigned long long* rare_count, int64_t* step, cudaStream_t st);

// Number this step's ionization products by the rank of their parent id.
// `done`: one zeroed counter per instance (left zeroed).
cudaError_t launch_births(const InstParams* inst, int ninst, Event* events,
                          unsigned long long* ev_count, unsigned long long* next_id,
                          uint32_t* id, uint32_t* keys_a, uint32_t* keys_b, unsigned* err,
                          cudaStream_t st);

// ---- sort (sort.cu) ---------------------------------------------------------------
struct SortArgs {
    const SegParams* seg;
    int nseg;
    int precision;
    const int64_t* tile_start;
    const int64_t* seg_nmove;
    unsigned long long* seg_n;
    unsigned long long* seg_live;
    unsigned long long* hwm_alt;      // slots in use of the other copy
    unsigned* hist;                   // per segment node arrays (cells), zeroed
    unsigned* tcount;                 // neutral targets: live targets per cell after the sort
                                      // (null: no target segment)
    int64_t seg_nodes;                // entries of the segment node arrays
    unsigned long long* newn;         // per segment live count after the sort
    unsigned long long* cell_part;    // per segment and chunk of 4096 cells: the chunk's count
    int cell_chunks;                  // chunks of the largest segment
    // source and destination stores
    int32_t* cell[2];
    void* off[2];
    void* ux[2];
    void* uy[2];
    void* uz[2];
    uint32_t* id[2];
    void* yp[2];                      // y coordinates of 2-D species (null: none)
    int src;
    int64_t max_cap;                  // largest segment capacity
    int max_cells;
    unsigned* err;                    // status word (the bounds-checked build's refusals)
};
// Grids are one resident wave of each kernel on `sms` multiprocessors.
cudaError_t launch_sort(const SortArgs& s, int nt, int sms, cudaStream_t st);
// The sort folded into a time step: the exclusive scan of the cell histogram the step
// before counted (`hist`, in place, and each segment's total into `newn`) before the
// sorting mover, and the new counts and the destination's empty tail after it.
cudaError_t launch_sort_scan(const SortArgs& s, cudaStream_t st);
cudaError_t launch_sort_finish(const SortArgs& s, cudaStream_t st);

// ---- I/O and diagnostics (io.cu) -------------------------------------------------
struct LoadArgs {
    const int32_t* cell;
    const void* off;        // double, or float with host_f32
    const void* vx;
    const void* vy;
    const void* vz;
    int host_f32;
    const uint32_t* id;     // NULL: id0 + k
    const uint8_t* state;   // collision clocks (own steps to skip, bit 7 pending), NULL: 0
    int64_t own0;           // the species' own index of its next moving step (clock origin)
    int64_t n;
    uint32_t id0;
    double vscale;          // dt/dx
    int64_t base, cap;
    int ncells;
    int32_t* s_cell;
    void* s_off;
    void* s_ux;
    void* s_uy;
    void* s_uz;
    uint32_t* s_id;
    void* s_yp;             // y coordinates (null: no 2-D species): set to 0
    unsigned* err;
    int precision;
    unsigned long long* next_id;  // instance's next automatic id: raised to max(id) + 1
};
cudaError_t launch_load(const LoadArgs& l, cudaStream_t st);
// clocks kept at their distance from each species' next moving step when the step
// counter is set from `from` to `to`
cudaError_t launch_rebase_clocks(const SegParams* seg, int nseg, int32_t* cell, int64_t from,
                                 int64_t to, cudaStream_t st);

struct GetArgs {
    const int32_t* s_cell;
    const void* s_off;
    const void* s_ux;
    const void* s_uy;
    const void* s_uz;
    const uint32_t* s_id;
    const void* s_yp;       // y coordinates (null: none)
    int64_t base, nslots;
    double vscale_inv;      // dx/dt
    int precision;
    int32_t* cell;
    void* off;              // double, or float with host_f32
    void* vx;
    void* vy;
    void* vz;
    int host_f32;
    uint32_t* id;
    uint8_t* state;         // collision clocks out, as own steps to skip (bit 7 pending)
    int64_t own0;           // the species' own index of its next moving step (clock origin)
    double* yp;             // y coordinates out (double), or null
    unsigned long long* block_count;  // scratch, ceil(nslots/1024)+1 entries
    int64_t capacity;                 // entries of the output arrays
    int64_t block0;                   // first 1024-slot block of this write launch
};
// Read-back in two phases: the live count of every 1024-slot block and their scan
// (block_count[b] = the output index of block b's first live particle, total at [nb]),
// then the compacted write of blocks [block0, block0 + nblocks), so that a caller can
// copy the output of one range to the host while the next range is written.
cudaError_t launch_get_scan(const GetArgs& g, cudaStream_t st);
cudaError_t launch_get_write(GetArgs g, int64_t block0, int64_t nblocks, cudaStream_t st);

// store yp[base + k] = in[k] (double in, the store's precision T), k < n
cudaError_t launch_set_yp(void* s_yp, int64_t base, const double* in, int64_t n, int precision,
                          cudaStream_t st);

// sum of kefac |u|^2 over live particles of segments [s0, s0+ns) into out[ns]
cudaError_t launch_kinetic(const SegParams* seg, int s0, int ns, int64_t max_slots,
                           const int32_t* cell, const void* ux, const void* uy,
                           const void* uz, int precision, double* out, cudaStream_t st);

cudaError_t launch_philox(uint64_t key, const uint32_t* ctr, uint32_t* out, int64_t n,
                          cudaStream_t st);

// fill int32 array p[lo, hi) with v
cudaError_t launch_fill_i32(int32_t* p, int64_t lo, int64_t hi, int32_t v, cudaStream_t st);

}  // namespace bitpic
