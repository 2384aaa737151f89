// Structure factors without a caller-provided workspace.
//
// Who needs this: some callers cannot call cudaMalloc (or any allocating
// routine) at the point where they want structure factors -- for example a
// plugin running inside a host application whose own caching allocator owns
// all device memory, or a real-time refinement loop that must not allocate
// after start-up because cudaMalloc can synchronise the device and take an
// unbounded time.  Such callers still own their inputs and outputs; only the
// scratch space of the structure-factor kernels is provided here, as a
// fixed-size array in device memory that the library reserves when it is
// loaded.
//
// Contract (also stated in include/fdx.h):
//   - the scratch is one file-scope __device__ array of FDX_NOALLOC_SF_SCRATCH_BYTES
//     (8 MiB); every GPU that loads libfdx keeps it until the process exits;
//   - sizes whose scratch does not fit are rejected with FDX_ERR_WORKSPACE
//     before any work is queued;
//   - the first call on a device looks up the array's device address on that
//     device (cudaGetSymbolAddress) and caches it; make that first call before
//     any stream capture;
//   - all calls share the one array and leave their partial sums in it; calls
//     whose work overlaps on the GPU (different streams, or different host
//     threads without ordering) race on it and must be serialised by the
//     caller;
//   - nothing in the scratch has to start at zero: every kernel writes each
//     scratch element it later reads within the same call.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fdx_internal.cuh"

using namespace fdx;

namespace {

constexpr size_t kScratchBytes = FDX_NOALLOC_SF_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_sf_scratch[kScratchBytes];

std::mutex g_mu;
void *g_ptr[kMaxDevices] = {nullptr};

// Device address of g_sf_scratch on the current device (looked up once per device).
int scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FDX_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sf_scratch) != cudaSuccess || !p) return FDX_ERR_CUDA;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return FDX_OK;
}

}  // namespace

extern "C" int fdx_structure_factors_noalloc(const fdx_cell *cell, const fdx_atoms *atoms,
                                             const fdx_broadening *br, int32_t n_refl, const int32_t *hkl,
                                             float *F_out, float *M_out, void *stream) {
    // the same argument checks, in the same order, as fdx_structure_factors
    int rc = validate_cell(cell);
    if (rc) return rc;
    if (!atoms || atoms->n_atoms < 1 || atoms->n_elem < 1 || atoms->n_elem > 64) return FDX_ERR_ARG;
    if (!atoms->frac || !atoms->B || !atoms->elem || !atoms->ff) return FDX_ERR_ARG;
    if (n_refl < 0) return FDX_ERR_ARG;
    if (n_refl > 0 && (!hkl || !F_out)) return FDX_ERR_ARG;
    if (br && (rc = validate_broadening(br))) return rc;
    if (n_refl == 0) return FDX_OK;

    // Scratch: packed atoms (uint4 + float2 each, element-sorted and padded),
    // the group list of the reflections (one int each) and one float4 partial
    // per (partial row, reflection).  Every element pass writes its own n_split
    // rows, so at least `passes` rows must fit; use the largest row budget
    // (at most 64) whose aligned layout fits the array.  sf_plan keeps
    // passes * n_split within that budget.
    const int passes = sf_passes(atoms->n_elem);
    int max_split = 64;
    while (max_split >= passes && sf_bind(nullptr, nullptr, atoms->n_atoms, n_refl, max_split) > kScratchBytes)
        --max_split;
    if (max_split < passes) return FDX_ERR_WORKSPACE;
    int n_split = 1, per = 1;
    sf_plan(atoms->n_atoms, n_refl, atoms->n_elem, max_split, n_split, per);
    if (passes * n_split > max_split) return FDX_ERR_WORKSPACE;  // never taken: sf_plan caps n_split

    void *base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;

    SFParams p;
    memset(&p, 0, sizeof p);
    double A[9], As[9];
    cell_basis(*cell, A, As);
    memcpy(p.As, As, sizeof As);
    p.n_atoms = atoms->n_atoms, p.n_elem = atoms->n_elem, p.n_refl = n_refl;
    p.n_split = n_split;
    p.frac = atoms->frac, p.B = atoms->B, p.occ = atoms->occ, p.ff = atoms->ff, p.elem = atoms->elem;
    sf_bind(&p, static_cast<char *>(base), atoms->n_atoms, n_refl, max_split);
    p.hkl = hkl, p.F_out = F_out, p.M_out = M_out;
    p.has_br = br ? 1 : 0;
    if (br) {
        p.intensity_model = br->intensity_model;
        for (int i = 0; i < 3; ++i) {
            p.g[i] = br->g[i], p.Bax[i] = br->B_axis[i];
            p.alen[i] = sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] + A[3 * i + 2] * A[3 * i + 2]);
        }
    }
    if (launch_structure_factors(p, static_cast<cudaStream_t>(stream)) != cudaSuccess) return FDX_ERR_CUDA;
    return FDX_OK;
}
