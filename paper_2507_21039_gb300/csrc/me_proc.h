// Internal (non-ABI) description of a generated process and its launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace me {

// Arguments of one |M|^2 launch.  All pointers are device pointers.
struct LaunchArgs {
    const double* mom;      // [nevt][npar][4] FP64
    long long nevt;
    double* me2;            // [nevt]
    double* hel_out;        // optional [nevt][nlist]: per-helicity contribution to me2
    const short* hel_list;  // helicity indices to sum (device)
    int nlist;
    int slots;              // lanes per event: power of two, <= 32
    double norm;            // g^{2k} / (IDEN * colour denominator)
    double mt;              // top mass (0 for massless fermions)
    int gauge_ext;          // -1, or external gluon whose polarisation is replaced by its momentum
    cudaStream_t stream;
    double* sde_w;          // optional [nevt]: single-diagram-enhancement weight of diagram sde_channel
    int sde_channel;
    const short* hel_ev;    // optional [nevt]: one sampled helicity per event (with nlist = 1, slots = 1)
    const double* w_ev;     // [nevt] with hel_ev: 1 / probability of the sampled helicity
    void* jscratch;         // optional: device memory for a launch's colour-flow scratch (kernels that
    size_t jscratch_bytes;  // keep J in global memory); the launch then allocates nothing and runs at
                            // most jscratch_bytes / jscratch_per_cta resident CTAs
};

enum Precision : int { PREC_FP64 = 0, PREC_FP32 = 1, PREC_MIXED = 2, PREC_MIXED64 = 3 };

struct ProcDesc {
    const char* name;
    int npar, nhel, ncol, ndiag, namp, ngluon, nlines, threads;
    double iden;               // initial spin x colour average x final identical-particle factor
    int cden;                  // colour-matrix denominator (C = num / cden)
    const int* cnum;           // colour numerators [ncol][ncol] (host)
    long long flops_hel;       // chain flops per evaluated helicity (generator count)
    long long colour_flops_hel;
    long long table_flops;     // per event, helicity-independent (the helicity-recycled tables)
    int coupling_power;        // |M|^2 proportional to (4 pi alpha)^coupling_power
    cudaError_t (*launch)(int precision, const LaunchArgs&);
    const int* diag_lines;     // [ndiag][4] internal-line masks of each diagram (host), 0-padded
    const int* diag_nlines;    // [ndiag]
    // bytes of global-memory colour-flow scratch one resident CTA of a launch in
    // this precision needs (0: the kernel keeps J on chip and allocates nothing)
    size_t (*jscratch_per_cta)(int precision);
    // resident CTAs of such a launch on the current device (its scratch is this x jscratch_per_cta)
    int (*jscratch_ctas)(int precision);
    int family;                // 0: e+e- -> mu+mu-, 1: g g -> t t~ + n g, 2: u u~ -> e+ e- + n g
};

const ProcDesc* find_process(const char* name);

}  // namespace me
