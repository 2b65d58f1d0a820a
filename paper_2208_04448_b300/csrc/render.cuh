// Ray marching through [Hash,5,4,NN(3)] (Section 4, the ray-marched Bunny Cloud): a pinhole
// camera, fixed steps along each ray inside the domain box, the density at every sample from
// the random-access query (trilinear over the regressed active corners, background
// elsewhere), and emission-absorption compositing front to back:
//   alpha_k = 1 - exp(-sigma rho_k dt),  L += T alpha_k rho_k,  T *= 1 - alpha_k.
// Samples are generated and composited in chunks of steps; the image holds (L, T) per pixel.
#pragma once
#include "common.cuh"

namespace nvdb {

struct RayCam {
  float eye[3], fwd[3], right[3], up[3];   // orthonormal basis; right / up scaled by the film extent
  float lo[3], hi[3];                       // domain box (index space)
  int width, height, max_steps;
  float step, sigma;
};

// Entry / exit distances of the ray of pixel (x, y) through the domain box (t_in > t_out: miss).
__device__ __forceinline__ void ray_box(const RayCam& c, int x, int y, float* dir, float& t_in, float& t_out) {
  const float u = (2.f * ((float)x + 0.5f) / (float)c.width - 1.f);
  const float v = (1.f - 2.f * ((float)y + 0.5f) / (float)c.height);
  float d[3], n2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d[a] = c.fwd[a] + u * c.right[a] + v * c.up[a];
    n2 = fmaf(d[a], d[a], n2);
  }
  const float inv = rsqrtf(n2);
  t_in = 0.f;
  t_out = 3.4e38f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dir[a] = d[a] * inv;
    if (dir[a] == 0.f) {   // parallel to this slab: inside it or a miss
      if (c.eye[a] < c.lo[a] || c.eye[a] > c.hi[a]) { t_in = 1.f; t_out = 0.f; }
      continue;
    }
    const float r = 1.f / dir[a];
    float t0 = (c.lo[a] - c.eye[a]) * r, t1 = (c.hi[a] - c.eye[a]) * r;
    if (t0 > t1) { const float tt = t0; t0 = t1; t1 = tt; }
    t_in = fmaxf(t_in, t0);
    t_out = fminf(t_out, t1);
  }
}

// Sample points of steps [s0, s0 + ns) of every ray: xyz[(ray * ns + k) * 3 ..], sample k at
// t_in + (s0 + k + 1/2) step; samples past the exit are placed outside the box (density 0).
__global__ void ray_points_kernel(RayCam c, int s0, int ns, float* xyz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nr = (int64_t)c.width * c.height;
  if (i >= nr * ns) return;
  const int64_t ray = i / ns;
  const int k = (int)(i % ns);
  float dir[3], t_in, t_out;
  ray_box(c, (int)(ray % c.width), (int)(ray / c.width), dir, t_in, t_out);
  const float t = t_in + ((float)(s0 + k) + 0.5f) * c.step;
  const bool inside = t_in <= t_out && t <= t_out;
#pragma unroll
  for (int a = 0; a < 3; ++a) xyz[3 * i + a] = inside ? fmaf(t, dir[a], c.eye[a]) : c.lo[a] - 4.f;
}

// Front-to-back compositing of the chunk's densities, one thread per ray, steps in order.
__global__ void ray_accum_kernel(RayCam c, int ns, const float* dens, float* img) {
  const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ray >= (int64_t)c.width * c.height) return;
  float L = img[2 * ray], T = img[2 * ray + 1];
  for (int k = 0; k < ns; ++k) {
    const float rho = fmaxf(dens[ray * ns + k], 0.f);
    const float alpha = 1.f - expf(-c.sigma * rho * c.step);
    L = fmaf(T * alpha, rho, L);
    T *= 1.f - alpha;
  }
  img[2 * ray] = L;
  img[2 * ray + 1] = T;
}

__global__ void ray_init_kernel(int64_t n, float* img) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { img[2 * i] = 0.f; img[2 * i + 1] = 1.f; }
}

}  // namespace nvdb
