// Host-side launchers shared by the C-ABI implementation (not part of the public ABI).
#pragma once
#include "pic_common.cuh"

namespace pic {

bool build_ttable(int l, int scheme, double dtt, TTable *t);
int ttable_eval_host(const TTable *t, int l, double delta, double *w);

// fused gather-push-deposit over all tiles of one run
cudaError_t launch_gpp(const RunDev &rd, int kt, cudaStream_t st);
size_t gpp_smem_bytes(const RunDev &rd);
// the 3D particle pass of either form (pic_gpp3d.cu); dynamic shared memory of its blocks
cudaError_t launch_gpp3d(const RunDev &rd, int kt, cudaStream_t st);
size_t gpp3d_smem_bytes(const RunDev &rd);

// Yee and grid kernels
cudaError_t launch_yee_b(const RunDev &rd, double h, bool shadow, cudaStream_t st);
cudaError_t launch_yee_e(const RunDev &rd, bool shadow, cudaStream_t st);
cudaError_t launch_shadow(const RunDev &rd, cudaStream_t st);

// particle packing (load / read back)
// particles p0 .. p0 + m - 1; x[a * xs + i], u[a * us + i] hold particle p0 + i
cudaError_t launch_pack(const RunDev &rd, int s, const double *x, int64_t xs, const double *u,
                        int64_t us, int64_t m, int64_t p0, cudaStream_t st);
// drifting plasma generated on the device: SplitMix64 stream keys of the offsets (per axis),
// the two Box-Muller uniforms of each momentum component and the flip uniform
struct LoadKeys {
    uint64_t pos[3];
    uint64_t mom[6];
    uint64_t flip;
    uint64_t jut[4];  // Sobol's method: the four uniforms of an attempt
    uint64_t dir[2];  // isotropic direction of a Juttner momentum
};
// theta > 0: Juttner-Synge co-moving momenta of temperature theta (u_th unused); else Gaussian
cudaError_t launch_load_plasma(const RunDev &rd, int s, const LoadKeys &keys, int64_t per_cell,
                               double gamma, double u_th, double theta, int64_t n, cudaStream_t st);
// particles p0 .. p0 + m - 1 -> x[a * m + i], u[a * m + i], cell[i]
cudaError_t launch_unpack(const RunDev &rd, int s, double *x, double *u, int64_t *cell,
                          int64_t m, int64_t p0, cudaStream_t st);

// diagnostics (device doubles): out[0] field energy sum, out[1] kinetic energy, out[2] max
// |D.E - rho|, out[3] max |G - gref| (gref != null), out[4] max continuity residual against
// rho_prev (rho_prev != null); rho receives the charge density of the current particles
cudaError_t launch_diag(const RunDev &rd, double *out, double *rho, const double *gref,
                        const double *rho_prev, cudaStream_t st);
// G = D.E - rho of the current state into gref (rho and 3 doubles of scratch overwritten)
cudaError_t launch_gauss_ref(const RunDev &rd, double *rho, double *gref, double *scratch,
                             cudaStream_t st);
// fixed-point current of a deterministic run -> FP64 (after the particle pass)
cudaError_t launch_det_finish(const RunDev &rd, cudaStream_t st);
// FP32 current of a 3D FP32 run (RunDev::J32) -> F[6..8] (after the particle pass)
cudaError_t launch_j32_finish(const RunDev &rd, cudaStream_t st);

// tile sort of one species
cudaError_t launch_sort(const RunDev &rd, int s, int64_t *tile_start, void *const *dst_pos,
                        void *const *dst_mom, int32_t *dst_cell, cudaStream_t st);

}  // namespace pic
