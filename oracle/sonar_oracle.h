/*
 * FP64 CPU oracle for per-ping coherent echo formation in a volumetric 3D sonar
 * ("Towards Realistic 3D Sonar Simulation", Sec. II.A-II.B and Sec. III, Eq. 1-3).
 *
 * TEST INFRASTRUCTURE ONLY. This library is loaded by tests/, by
 * __graft_entry__.smoke() and by bench.py's cpu_baseline leg, never by the product
 * path. It shares no code, header, table or constant with the CUDA library.
 *
 * The paper proposes the method without formulas; every formula here is a reading of
 * Sec. II (ray casting, Snell refraction, per-hit backscatter, speckle, limited
 * secondary reflections, complex baseband accumulation with delay-set phase and
 * coherent summation into beams), stated next to the function that implements it.
 *
 * Parity unpinned (no closed form or brute force fixes them): Lambertian amplitudes
 * on meshes, speckle statistics, multi-bounce mesh routes, curved-ray mesh hits.
 */
#ifndef SONAR_ORACLE_H
#define SONAR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t nx, ny;          /* receive array elements along y (nx) and z (ny) */
  double pitch;            /* element pitch [m] */
  double f0, bw, pulse;    /* carrier [Hz], chirp bandwidth [Hz], pulse length T_p [s] */
  double c_ref;            /* reference sound speed; <= 0 means c(z_sonar) */
  double hfov, vfov;       /* fields of view [rad] */
  int32_t n_beam_az, n_beam_el, n_range;
  double r_min, r_max, r_blank;
  int32_t n_ray_az, n_ray_el, n_sub;   /* ray grid; n_sub in {1, 4} */
  int32_t max_bounces;
  double surface_z;        /* NaN: no sea surface */
  double r_surface, r_seabed;
  double alpha;            /* amplitude attenuation [Np/m] */
  uint64_t seed;
  int32_t thr_mode;        /* 0 absolute, 1 relative to the ping maximum */
  double thr;
  int32_t cross;           /* 1: add out/back cross-term multipath (isovelocity only) */
  int64_t vol_n;           /* water-column scatterers (0: none; isovelocity only) */
  double vol_lo[3], vol_hi[3];  /* their world-frame box [m] */
  double vol_sv;           /* volume backscattering coefficient s_v [1/m] */
  int32_t fld_nx, fld_nz;  /* range-dependent sound speed c(x, z) on a grid (0: none) */
  double fld_x0, fld_dx, fld_z0, fld_dz;  /* grid origin and spacing [m] */
  const double* fld_c;     /* [fld_nz][fld_nx] sound speed [m/s] */
  double fld_h;            /* ray integration step in arc length [m] */
} orc_params;

typedef struct {
  int64_t n_verts; const float* verts;      /* [n_verts][3] */
  int64_t n_tris; const int32_t* tris;      /* [n_tris][3] */
  const float* mu;                          /* [n_tris] backscatter coefficient */
  const uint8_t* flags;                     /* [n_tris] bit0: specular mirror */
  int64_t n_points; const float* points;    /* [n_points][3] */
  const float* sigma;                       /* [n_points] amplitude coefficient */
  int64_t n_planes; const double* planes;   /* [n_planes][4]: unit normal, offset (n.x = d) */
} orc_scene;

typedef struct {
  int64_t cap, n;
  int32_t *ray, *sub, *seg, *prim;   /* points: ray = point index, sub = route, prim = -1 */
  double *tau, *len, *amp, *psi, *phi;  /* two-way delay, one-way path length, |c|, speckle, arg c */
  double *ux, *uy, *uz;              /* sensor-frame arrival direction */
  double *cr, *ci;                   /* complex coefficient c_k */
  double *margin, *gap;              /* barycentric margin and distance gap to the runner-up */
  double *kinc, *gam;                /* mesh hits: incidence cosine |d . n| at the facet and the
                                        route's one-way reflection product; 0 for other hits */
  double c_ref;                      /* resolved reference sound speed (output) */
} orc_hits;

/* Normalised autocorrelation R(u) of the Hann-windowed LFM pulse. */
void orc_pulse_acf(double u, double pulse, double bw, double* re, double* im);
/* OpenMP threads of the parallel loops (n > 0). */
void orc_set_threads(int n);
/* The transmitted pulse p(t): Hann-windowed linear chirp over |t| <= T/2. */
void orc_pulse(double t, double pulse, double bw, double* re, double* im);

/* 32-bit pcg4d hash (Jarzynski & Olano 2020); v is updated in place. */
void orc_pcg4d(uint32_t v[4]);

/* Closest-hit query: returns prim (or -1); t, u, v of the hit; runner-up distance. */
int32_t orc_closest_hit(const orc_scene* sc, const double o[3], const double d[3],
                        double tmin, double tmax, int32_t exclude, int use_bvh,
                        double* t, double* margin, double* t_second);

/* Test access to the field-route integrator: n RK4 steps of arc length h from the point
   o along the unit direction d in the sound-speed field of p; out = (r[3], t[3], T), the
   position, unit tangent and one-way time. Returns 0, or 5 for an invalid field. */
int orc_field_ray(const orc_params* p, const double o[3], const double d[3], double h, int32_t n, double out[7]);

/* Trace one ping: fills the hit list. Returns 0, or -needed when capacity is short,
   or a positive error code. */
int orc_trace(const orc_scene* sc, const orc_params* p, const double pose_t[3],
              const double pose_q[4], const double* ssp_z, const double* ssp_c,
              int32_t n_ssp, int use_bvh, orc_hits* out);

/* Element echoes s_m[n] for samples ns[0..n_ns): out[n_ns][M][2]. */
/* Raw element series at t_n + s dt / U (the echo before pulse compression). */
void orc_raw(const orc_params* p, const orc_hits* h, int32_t U, int32_t s, const int32_t* ns, int64_t n_ns,
             double* s_out);
void orc_synth(const orc_params* p, const orc_hits* h, const int32_t* ns, int64_t n_ns,
               double* s_out);

/* Wideband element echoes (plane-wave delay u_k . p_m / c in the envelope and the phase)
   at t_n + shift: out[n_ns][M][2]. */
void orc_synth_wb(const orc_params* p, const orc_hits* h, double shift, const int32_t* ns, int64_t n_ns,
                  double* s_out);
/* True-time-delay beamforming of the wideband echoes, exact in time, from the hits:
   b_out[n_beams][n_ns][2]. */
void orc_ttd(const orc_params* p, const orc_hits* h, const float* taper, const int32_t* ns, int64_t n_ns,
             const int32_t* beams, int64_t n_beams, double* b_out);

/* Beams B[b][i] = sum_m w_m e^{-j k u_b.p_m} s_m[ns_i] / sum w, for beams[0..n_beams). */
void orc_beamform(const orc_params* p, double c_ref, const float* taper,
                  const double* s, int64_t n_ns, const int32_t* beams, int64_t n_beams,
                  double* b_out);

/* Envelope E[b][i] = |B[b][i]| * TVG(r_{ns_i}). */
void orc_envelope(const orc_params* p, const double* b, const int32_t* ns, int64_t n_ns,
                  int64_t n_beams, double* e_out);

/* Point cloud from a full envelope volume E[Nb][Nr]. Writes up to Nb points
   (x, y, z, intensity, beam, bin) and returns the count. */
int64_t orc_peaks(const orc_params* p, const double pose_t[3], const double pose_q[4],
                  const double* e, double* pts_xyzi, int32_t* pts_beam, int32_t* pts_bin);

/* Curved-ray marching in a linear sound-speed profile: from position o with launch
   direction d (unit), returns n_nodes arc nodes at spacing h (positions, one-way
   times, grazing angles). */
void orc_arc_nodes(const double* ssp_z, const double* ssp_c, int32_t n_ssp,
                   const double o[3], const double d[3], double h, int32_t n_nodes,
                   double* pos, double* times, double* theta);

/* Eigen-arc from o to x in a linear profile: launch direction (world), one-way time,
   arc length. Returns 0 on success. */
int orc_eigen_arc(const double* ssp_z, const double* ssp_c, int32_t n_ssp,
                  const double o[3], const double x[3], double d_out[3],
                  double* t_out, double* s_out);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
