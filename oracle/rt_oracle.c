/*
 * rt_oracle.c -- plain, slow, FP64 CPU oracle for photon-conserving adaptive
 * ray tracing (Wise & Abel, "Enzo+Moray", arXiv:1012.2865).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker that the CUDA path is
 * compared against.  It shares no code with the CUDA library and must never be
 * called by the product path; only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.
 *
 * It follows the paper's statement of the method, in the paper's order:
 *   Sec. 2.1  adaptive ray tracing: HEALPix emission (N_pix = 12 * 4^l), the
 *             next-crossing distance (Eq. "trace"), the split test (Eq.
 *             "split") with children p' = 4p + {0,1,2,3} carrying P/4 from
 *             the parent's radius, and the termination conditions;
 *   Sec. 2.2  segment optical depth (Eq. "dtau"), photon-conserving absorption
 *             (Eq. "flux"), the photo-ionisation / photo-heating deposits
 *             (Eqs. "kph", "gamma") and the hydrogen-only rate equation
 *             (Eq. "dndt");
 *   Sec. 3.1  Steps 1-6 (create packages, zero fields, trace each package,
 *             chemistry on the irradiated state).
 *
 * Readings where the paper is silent or garbled (each one also listed in the
 * design notes of the repository):
 *   R1 Eq. "trace" as printed gives a negative length; the segment length is
 *      dr = min_i t_i - r, t_i the distance from the source to the next cell
 *      plane along the ray on axis i (Step 3d).
 *   R2 The split test uses the radius at the END of the segment, r + dr
 *      (Step 3e): split when r_next > R_split(l) = sqrt(N_pix(l)/(4 pi Phi_c))
 *      cell widths, decided before the cell is traversed; the children start
 *      at the parent's current radius.  No split beyond max_level.
 *   R3 Termination "P below f_term of its initial value": because children
 *      inherit both P/4 and the accumulated optical depth, this is
 *      tau_tot > -ln(f_term).  The residual P is absorbed in the current cell
 *      so that emitted = absorbed + escaped holds exactly.
 *   R4 Cell of a point lying on a cell plane: along an axis with n_i > 0 take
 *      floor(u), with n_i < 0 take ceil(u) - 1, with n_i == 0 take floor(u).
 *   R5 k_ph written in the form P sigma dr phi(tau) / V with
 *      phi(tau) = (1 - e^-tau)/tau (phi(0) = 1), which equals Eq. "kph" for
 *      n_abs > 0 and is its limit at n_abs = 0.  P is in photons per second,
 *      so the dt_P of Eq. "kph" cancels.
 *   R6 Eq. "dndt" lacks the n_HI factor on the k_ph term; the ionisation term
 *      is k_ph n_HI.  Hydrogen only: n_e = n_p = n_H (1 - x_HI); C_H = 0.
 *   R7 The implicit x_HI update is backward Euler with nsub equal substeps,
 *      k_ph frozen over the step (operator split, Step 6).
 *   R8 Pixel directions use an exact quadrant reduction of the azimuth so that
 *      components that vanish are exactly 0 and mirror-symmetric pixels give
 *      mirror-symmetric vectors.
 *  R13 Covering factor (Sec. 2.3, optional): R_0 in L_pix = R_0 theta_pix is
 *      the radius where the segment starts; theta_pix = sqrt(Omega_pix) of a
 *      square pixel; f_c is capped at 1 ("pixel fully contained") and is 1 at
 *      r = 0; it scales every k_ph / Gamma contribution of the segment,
 *      including the residual absorbed at termination (R3), never dP.
 *  R15 Finite speed of light (Sec. 2.1 halting condition 1, Step 3j,
 *      optional): a package may travel c dt_P per trace beyond the radius
 *      at which its lineage entered the trace, so a package emitted a traces
 *      ago halts at rlim[a] = c dt_P summed over the a + 1 traces since its
 *      emission (same FP64 sum on both sides: rlim'[0] = c dt_P,
 *      rlim'[a] = rlim[a - 1] + c dt_P).  The test follows the split test and
 *      uses the crossing radius of the cell: when r_next > rlim the segment
 *      ends at rlim, is absorbed as usual (termination is checked first),
 *      and the package is kept with its cell; the next trace continues it
 *      from that radius and cell through the then current medium.  Children
 *      inherit the age.  Emitted + resumed = absorbed + escaped + halted.
 *  R16 Photon types (Sec. 3.2, optional): a source emits packages of one
 *      type -- H I, He I or He II ionising -- and a package of a type is
 *      absorbed by that type's absorber only (Eq. "dtau" with its n_abs;
 *      n_HI = n_H x_HI, n_HeI and n_HeII given per cell), deposits into that
 *      type's k_ph and Gamma, and heats with E_ph - E_i, E_i = 13.6, 24.6,
 *      54.4 eV.  The helium network that would use these rates is not part
 *      of the method's hot path; the update stays hydrogen-only.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (no FMA
 * contraction, so the rounding of every expression is the one written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EV_ERG 1.602176634e-12 /* erg per eV (exact by definition) */
#define ORC_E_HI 13.6              /* hydrogen ionisation threshold, eV (Sec. 2.2) */
#define ORC_MAX_LEVEL 14           /* pixel numbers at level 14 still fit 32 bits */
#define ORC_NTYPES 3               /* photon types: H I, He I, He II ionising (Sec. 3.2) */
/* ionisation energies of the absorbers of the photon types, eV (reading R16) */
static const double orc_e_ion[ORC_NTYPES] = {ORC_E_HI, 24.6, 54.4};

/* ------------------------------------------------------------------------- */
/* HEALPix, nested scheme (Gorski et al. 2005), written from the projection   */
/* geometry.  Face f in 0..11: 0-3 north, 4-7 equatorial, 8-11 south.  In the */
/* projection plane (t = 4 phi / pi, u = 3z/2 in the equatorial belt), face    */
/* centres are (2k+1, 1) north, (2k, 0) equatorial, (2k+1, -1) south, and a    */
/* pixel (ix, iy) of a face sits at p1 = (ix+1/2)/Nside, p2 = (iy+1/2)/Nside   */
/* along the two diagonals: dt = p1 - p2, du = p1 + p2 - 1.                    */
/* ------------------------------------------------------------------------- */

static uint32_t orc_compact_bits(uint64_t v) {
  /* gather the even-position bits of v into the low half */
  uint32_t out = 0;
  for (int b = 0; b < 32; ++b) out |= (uint32_t)((v >> (2 * b)) & 1u) << b;
  return out;
}

static uint64_t orc_spread_bits(uint32_t v) {
  uint64_t out = 0;
  for (int b = 0; b < 32; ++b) out |= (uint64_t)((v >> b) & 1u) << (2 * b);
  return out;
}

/* Ring-scheme description of a nested pixel: z (exact rational, correctly
 * rounded), 1 - |z| where it is needed for accuracy near the poles, and the
 * azimuth phi = (pi/2) * a / b with integers a, b. */
static void orc_pixel_ring(int level, uint64_t pix, double *z, double *sin_theta,
                           int64_t *a, int64_t *b) {
  const int64_t nside = (int64_t)1 << level;
  const uint64_t npface = (uint64_t)nside * (uint64_t)nside;
  const int face = (int)(pix / npface);
  const uint64_t ipf = pix % npface;
  const int64_t ix = orc_compact_bits(ipf);
  const int64_t iy = orc_compact_bits(ipf >> 1);
  const int64_t s = ix + iy + 1;
  const int k = face & 3;
  int64_t nr;            /* pixels per quadrant in the ring of this pixel */
  int64_t tnum;          /* t * nr, with t = 4 phi / pi at the pixel centre */
  if (face < 4) {        /* north face, centre (2k+1, 1) */
    if (s > nside) {     /* polar cap: sigma = 2 - u = nr / nside */
      nr = 2 * nside - s;
      double omz = (double)(nr * nr) / (double)(3 * nside * nside);
      *z = 1.0 - omz;
      *sin_theta = sqrt(omz * (2.0 - omz));
    } else {
      nr = nside;
      *z = (double)(2 * s) / (double)(3 * nside);
      *sin_theta = sqrt((1.0 - *z) * (1.0 + *z));
    }
    tnum = (2 * k + 1) * nr + ix - iy;
  } else if (face < 8) { /* equatorial face, centre (2k, 0) */
    nr = nside;
    *z = (double)(2 * (s - nside)) / (double)(3 * nside);
    *sin_theta = sqrt((1.0 - *z) * (1.0 + *z));
    tnum = 2 * k * nr + ix - iy;
  } else {               /* south face, centre (2k+1, -1) */
    if (s < nside) {
      nr = s;
      double omz = (double)(nr * nr) / (double)(3 * nside * nside);
      *z = -(1.0 - omz);
      *sin_theta = sqrt(omz * (2.0 - omz));
    } else {
      nr = nside;
      *z = (double)(2 * (s - 2 * nside)) / (double)(3 * nside);
      *sin_theta = sqrt((1.0 - *z) * (1.0 + *z));
    }
    tnum = (2 * k + 1) * nr + ix - iy;
  }
  /* phi = (pi/4) * tnum / nr = (pi/2) * tnum / (2 nr); wrap into [0, 2 pi) */
  int64_t bb = 2 * nr;
  int64_t aa = tnum % (4 * bb);
  if (aa < 0) aa += 4 * bb;
  *a = aa;
  *b = bb;
}

/* (cos phi, sin phi) for phi = (pi/2) * a / b, 0 <= a < 4b, with the
 * quadrant removed exactly (R8). */
static void orc_cos_sin_quarter(int64_t a, int64_t b, double *c, double *s) {
  int64_t q = a / b;
  int64_t m = a - q * b; /* 0 <= m < b: angle (pi/2) m / b inside the quadrant */
  double c0, s0;
  if (m == 0) {
    c0 = 1.0;
    s0 = 0.0;
  } else if (2 * m == b) {
    c0 = sqrt(0.5);
    s0 = c0;
  } else if (2 * m < b) {
    double ang = (M_PI * 0.5) * ((double)m / (double)b);
    c0 = cos(ang);
    s0 = sin(ang);
  } else {
    double ang = (M_PI * 0.5) * ((double)(b - m) / (double)b);
    c0 = sin(ang);
    s0 = cos(ang);
  }
  switch (q) {
    case 0: *c = c0; *s = s0; break;
    case 1: *c = -s0; *s = c0; break;
    case 2: *c = -c0; *s = -s0; break;
    default: *c = s0; *s = -c0; break;
  }
}

/* Step 3a: unit vector of the centre of nested pixel `pix` at `level`. */
void orc_pix2vec_nest(int level, uint64_t pix, double v[3]) {
  double z, st, c, s;
  int64_t a, b;
  orc_pixel_ring(level, pix, &z, &st, &a, &b);
  orc_cos_sin_quarter(a, b, &c, &s);
  v[0] = st * c;
  v[1] = st * s;
  v[2] = z;
}

/* (z, phi) of a pixel centre, phi in [0, 2 pi); for tests of the ring layout. */
void orc_pix2ang_nest(int level, uint64_t pix, double *z, double *phi) {
  double st;
  int64_t a, b;
  orc_pixel_ring(level, pix, z, &st, &a, &b);
  *phi = (M_PI * 0.5) * ((double)a / (double)b);
}

/* Inverse map: direction (z, phi) -> nested pixel, from the same projection. */
uint64_t orc_ang2pix_nest(int level, double z, double phi) {
  const int64_t nside = (int64_t)1 << level;
  double t = phi / (M_PI * 0.25); /* t = 4 phi / pi */
  t = fmod(t, 8.0);
  if (t < 0) t += 8.0;
  double za = fabs(z);
  int face;
  double dt, du;
  if (za > 2.0 / 3.0) {
    double sigma = sqrt(3.0 * (1.0 - za));
    int k = (int)floor(t * 0.5);
    if (k > 3) k = 3;
    double tc = 2.0 * k + 1.0;
    dt = (t - tc) * sigma;
    if (z > 0) { face = k; du = 1.0 - sigma; }
    else { face = k + 8; du = sigma - 1.0; }
  } else {
    double u = 1.5 * z;
    double ce = 2.0 * floor(t * 0.5 + 0.5); /* nearest even t: equatorial centre */
    double dte = t - ce;
    if (fabs(dte) + fabs(u) <= 1.0) {
      face = 4 + ((int)ce / 2) % 4;
      dt = dte;
      du = u;
    } else {
      int k = (int)floor(t * 0.5);
      if (k > 3) k = 3;
      double tc = 2.0 * k + 1.0;
      dt = t - tc;
      if (u > 0) { face = k; du = u - 1.0; }
      else { face = k + 8; du = u + 1.0; }
    }
  }
  double p1 = 0.5 * (du + dt + 1.0), p2 = 0.5 * (du - dt + 1.0);
  int64_t ix = (int64_t)floor(p1 * (double)nside);
  int64_t iy = (int64_t)floor(p2 * (double)nside);
  if (ix < 0) ix = 0;
  if (ix > nside - 1) ix = nside - 1;
  if (iy < 0) iy = 0;
  if (iy > nside - 1) iy = nside - 1;
  return (uint64_t)face * (uint64_t)(nside * nside) + orc_spread_bits((uint32_t)ix) +
         (orc_spread_bits((uint32_t)iy) << 1);
}

/* ------------------------------------------------------------------------- */
/* Geometry of one ray in cell units (cell width = 1).                        */
/* ------------------------------------------------------------------------- */

/* R4: index of the cell holding coordinate u along an axis with direction n. */
static int64_t orc_cell_of(double u, double n) {
  if (n > 0) return (int64_t)floor(u);
  if (n < 0) return (int64_t)ceil(u) - 1;
  return (int64_t)floor(u);
}

static int orc_inside(const int64_t c[3], const int dims[3]) {
  return c[0] >= 0 && c[0] < dims[0] && c[1] >= 0 && c[1] < dims[1] && c[2] >= 0 &&
         c[2] < dims[2];
}

/* Step 3b: cell of the point s + r n. */
static void orc_locate(const double s[3], const double n[3], double r, int64_t c[3]) {
  for (int i = 0; i < 3; ++i) c[i] = orc_cell_of(s[i] + r * n[i], n[i]);
}

/* Step 3d / Eq. "trace" (reading R1): distance from the source to the next
 * cell plane on each axis, and the smallest of them. */
static double orc_next_crossing(const double s[3], const double n[3], const int64_t c[3],
                                double t[3]) {
  double tmin = INFINITY;
  for (int i = 0; i < 3; ++i) {
    if (n[i] > 0) t[i] = ((double)(c[i] + 1) - s[i]) / n[i];
    else if (n[i] < 0) t[i] = ((double)c[i] - s[i]) / n[i];
    else t[i] = INFINITY;
    if (t[i] < tmin) tmin = t[i];
  }
  return tmin;
}

/* Move into the next cell: every axis whose plane is reached at r_next steps. */
static void orc_advance(const double n[3], const double t[3], double rnext, int64_t c[3]) {
  for (int i = 0; i < 3; ++i)
    if (n[i] != 0 && t[i] == rnext) c[i] += (n[i] > 0) ? 1 : -1;
}

/* Cell sequence of one unsplit ray from radius r0 until it leaves the box:
 * cell index triples and segment lengths (cell units).  Returns the number of
 * segments written (at most max_out), including zero-length ones. */
int orc_ray_path(const int dims[3], const double s[3], const double n[3], double r0, int max_out,
                 int64_t *cells /* 3*max_out */, double *dr_out, double *r_out) {
  int64_t c[3];
  double t[3];
  double r = r0;
  int cnt = 0;
  orc_locate(s, n, r, c);
  while (orc_inside(c, dims) && cnt < max_out) {
    double rnext = orc_next_crossing(s, n, c, t);
    double dr = rnext - r;
    if (dr < 0) dr = 0;
    cells[3 * cnt + 0] = c[0];
    cells[3 * cnt + 1] = c[1];
    cells[3 * cnt + 2] = c[2];
    dr_out[cnt] = dr;
    r_out[cnt] = r;
    ++cnt;
    orc_advance(n, t, rnext, c);
    r = rnext;
  }
  return cnt;
}

/* ------------------------------------------------------------------------- */
/* Compensated (Neumaier) summation for the FP64 photon budget.               */
/* ------------------------------------------------------------------------- */
typedef struct { double sum, comp; } orc_ksum;

static void orc_kadd(orc_ksum *k, double v) {
  double t = k->sum + v;
  if (fabs(k->sum) >= fabs(v)) k->comp += (k->sum - t) + v;
  else k->comp += (v - t) + k->sum;
  k->sum = t;
}

static double orc_kval(const orc_ksum *k) { return k->sum + k->comp; }

/* Order-independent checksum of the set of created packages (source, level,
 * pixel): sum over packages of a 64-bit mix, taken modulo 2^64. */
static uint64_t orc_pkg_hash(uint32_t src, uint32_t level, uint64_t pix) {
  uint64_t x = ((uint64_t)src << 40) ^ ((uint64_t)level << 34) ^ pix;
  x ^= x >> 31;
  x *= 0x7fb5d329728ea185ULL;
  x ^= x >> 27;
  x *= 0x81dadef4bc2dd44dULL;
  x ^= x >> 33;
  return x;
}

/* ------------------------------------------------------------------------- */
/* The trace: Steps 1-5 for every source of one grid.                         */
/* ------------------------------------------------------------------------- */
typedef struct {
  uint32_t src, level;
  uint64_t pix;
  double r;   /* distance travelled, cell units */
  double P;   /* photons per second carried */
  double tau; /* optical depth accumulated by the package and its ancestors */
  uint32_t age;     /* traces since the lineage was emitted (R15) */
  int has_cell;     /* resumed package: continue in cell[] (R15) */
  int64_t cell[3];
} orc_pkg;

/* A package halted by the finite speed of light (R15), as kept between
 * traces: its state, the cell it halted in, and its age in the next trace. */
typedef struct {
  uint32_t src, level;
  uint64_t pix;
  double r, P, tau;
  int64_t cell[3];
  uint32_t age;
  uint32_t pad;
} orc_flight;

typedef struct {
  orc_pkg *v;
  size_t n, cap;
} orc_stack;

static int orc_push(orc_stack *st, orc_pkg p) {
  if (st->n == st->cap) {
    size_t nc = st->cap ? 2 * st->cap : 1024;
    orc_pkg *nv = (orc_pkg *)realloc(st->v, nc * sizeof(orc_pkg));
    if (!nv) return -1;
    st->v = nv;
    st->cap = nc;
  }
  st->v[st->n++] = p;
  return 0;
}

/* Eq. "fc" (Sec. 2.3): the covering factor of a segment, reading R13.  The
 * pixel is taken as a square of width L_pix = r theta_pix (theta_pix =
 * sqrt(4 pi / N_pix), r the radius where the segment starts) centred on the
 * segment's midpoint; D_edge is the distance from the midpoint to the
 * nearest face of the cell along the three axes, dx/2 - max_i D_c,i (Eq.
 * "midpoint"); f_c = (1/2 + D_edge / L_pix)^2, and 1 where the pixel fits in
 * the cell (f_c > 1) or has no width (r = 0).  Cell units throughout. */
static double orc_fc(const double s[3], const double n[3], double r, double dr, const int64_t c[3],
                     double theta_pix) {
  const double L = r * theta_pix;
  if (!(L > 0)) return 1.0;
  double dmax = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double mid = s[i] + n[i] * (r + 0.5 * dr);
    const double d = fabs(mid - ((double)c[i] + 0.5));
    if (d > dmax) dmax = d;
  }
  const double f = 0.5 + (0.5 - dmax) / L;
  return f * f < 1.0 ? f * f : 1.0;
}

/* Everything one trace needs while it walks packages. */
typedef struct {
  const int *dims;
  size_t ncell;
  const double *n_abs;     /* absorber density per photon type and cell: [type][cell] (R16) */
  const int *type;         /* photon type per source (NULL: all H I) */
  double dx, vol, tau_term;
  const double *rsplit;
  int max_level, fc, src_offset;
  const double *s;         /* source positions, cell units, 3 per source */
  const double *sigma_cm2;
  const double *heat;      /* (E_ph - 13.6 eV) in erg per source */
  int n_ages;              /* 0: infinite speed of light */
  const double *rlim;      /* halting radius per age (R15), cell units */
  double *kph, *gamma;
  uint64_t *counts, *hashes, nseg;
  orc_ksum absorbed, escaped, halted;
  orc_flight *out;
  size_t out_cap, n_out;
} orc_run;

/* Steps 3a-3k for every package on the stack and its descendants, until each
 * is split, absorbed, gone or halted.  Returns -1 on an allocation failure or
 * a package whose age has no halting radius. */
static int orc_walk(orc_run *R, orc_stack *st) {
  const int *dims = R->dims;
  while (st->n > 0) {
    orc_pkg pk = st->v[--st->n];
    const double *s = R->s + 3 * pk.src;
    const double sigma_dx = R->sigma_cm2[pk.src] * R->dx;
    const size_t toff = R->type ? (size_t)R->type[pk.src] * R->ncell : 0; /* R16 */
    const double *n_abs = R->n_abs + toff;
    double *kph = R->kph + toff, *gamma = R->gamma + toff;
    double rlim = INFINITY;
    if (R->n_ages > 0) {
      if (pk.age >= (uint32_t)R->n_ages) return -1;
      rlim = R->rlim[pk.age];
    }
    double n[3];
    orc_pix2vec_nest((int)pk.level, pk.pix, n); /* Step 3a */
    int64_t c[3];
    if (pk.has_cell) { c[0] = pk.cell[0]; c[1] = pk.cell[1]; c[2] = pk.cell[2]; }
    else orc_locate(s, n, pk.r, c); /* Step 3b */
    for (;;) {
      if (!orc_inside(c, dims)) { /* Step 3k, isolated boundaries */
        orc_kadd(&R->escaped, pk.P);
        break;
      }
      double t[3];
      double rnext = orc_next_crossing(s, n, c, t); /* Step 3d */
      if ((int)pk.level < R->max_level && rnext > R->rsplit[pk.level]) { /* Step 3e */
        for (int kk = 3; kk >= 0; --kk) {
          orc_pkg ch = {pk.src, pk.level + 1, 4 * pk.pix + (uint64_t)kk, pk.r, pk.P / 4.0, pk.tau,
                        pk.age, 0, {0, 0, 0}};
          if (orc_push(st, ch)) return -1;
          R->counts[pk.level + 1] += 1;
          R->hashes[pk.level + 1] +=
              orc_pkg_hash(pk.src + (uint32_t)R->src_offset, pk.level + 1, 4 * pk.pix + (uint64_t)kk);
        }
        break;
      }
      /* Step 3j (reading R15): the segment ends where the package has
       * travelled c dt_P since its lineage's emission */
      double rend = rnext;
      int halt = 0;
      if (rnext > rlim) { rend = rlim; halt = 1; }
      double dr = rend - pk.r;
      if (dr < 0) dr = 0;
      const size_t idx = (size_t)c[0] + (size_t)dims[0] * ((size_t)c[1] + (size_t)dims[1] * (size_t)c[2]);
      /* Step 3f: Eqs. "dtau", "flux", "kph" (reading R5), "gamma" */
      const double dtau = sigma_dx * n_abs[idx] * dr;
      const double absorbed_frac = -expm1(-dtau);         /* 1 - e^-tau */
      const double dP = pk.P * absorbed_frac;
      const double phi = (dtau > 0) ? absorbed_frac / dtau : 1.0;
      const double f_c =
          R->fc ? orc_fc(s, n, pk.r, dr, c, sqrt(4.0 * M_PI / (12.0 * ldexp(1.0, 2 * (int)pk.level)))) : 1.0;
      const double k_add = pk.P * R->sigma_cm2[pk.src] * (dr * R->dx) * phi / R->vol * f_c;
      kph[idx] += k_add;
      gamma[idx] += k_add * R->heat[pk.src];
      if (dr > 0) ++R->nseg;
      /* Step 3h */
      pk.P -= dP;
      pk.tau += dtau;
      orc_kadd(&R->absorbed, dP);
      /* Step 3i (reading R3): absorb the residual in this cell */
      if (pk.tau > R->tau_term) {
        const double k_res = pk.P / (n_abs[idx] * R->vol) * f_c;
        kph[idx] += k_res;
        gamma[idx] += k_res * R->heat[pk.src];
        orc_kadd(&R->absorbed, pk.P);
        break;
      }
      if (halt) { /* Step 3j: keep the package for the next trace */
        if (R->n_out < R->out_cap) {
          orc_flight f = {pk.src, pk.level, pk.pix, rend, pk.P, pk.tau, {c[0], c[1], c[2]}, pk.age + 1, 0};
          R->out[R->n_out] = f;
        }
        R->n_out++;
        orc_kadd(&R->halted, pk.P);
        break;
      }
      orc_advance(n, t, rnext, c);
      pk.r = rnext;
    }
  }
  return 0;
}

/*
 * orc_trace_mf: one radiative-transfer pass over a uniform grid.
 *   dims        nx, ny, nz (cells); cell index = i + nx*(j + ny*k)
 *   box_len_cm  length of the x extent; cell width dx = box_len_cm / nx
 *   n_H, x_HI   hydrogen density (cm^-3) and neutral fraction per cell
 *   n_he        NULL, or [2*ncell]: n_HeI then n_HeII per cell (cm^-3), the
 *               absorbers of the He I and He II photon types (R16)
 *   nsrc, pos_cm[3*nsrc], ndot[nsrc] (photons/s), e_ph_eV[nsrc],
 *   sigma_cm2[nsrc]
 *   src_type    NULL (all H I), or [nsrc] photon type 0, 1, 2 (R16; types
 *               1 and 2 need n_he)
 *   level0, phi_c, f_term, max_level   method parameters (Sec. 2.1)
 *   fc           nonzero: scale the k_ph and Gamma contributions by the
 *                covering factor of Eq. "fc" (photon budget unchanged)
 *   src_offset   index of the first source in the checksum (a shard of a
 *                larger source list hashes its sources as the whole list does)
 *   n_ages, rlim[n_ages]   halting radius per age in cell units (R15);
 *                n_ages = 0: infinite speed of light
 *   n_in, in[n_in]         packages halted by the previous trace, resumed
 *                          here (photons/s as they were emitted)
 *   out_cap, out           room for the packages this trace halts
 * outputs (overwritten):
 *   kph[nt*ncell]   photo-ionisation rate per absorber, s^-1 (Eq. "kph"),
 *                   per photon type (nt = 3 with n_he, else 1)
 *   gamma[nt*ncell] photo-heating rate per absorber, erg/s (Eq. "gamma")
 *   budget[5]    emitted, absorbed, escaped, resumed, halted photons/s
 *                (Neumaier sums)
 *   counts[ORC_MAX_LEVEL+1]   packages created per level
 *   hashes[ORC_MAX_LEVEL+1]   checksum of the created (src, level, pixel) set
 *   segments     number of segments with dr > 0
 *   n_out        packages halted (when above out_cap, only out_cap stored)
 * returns 0; -1 on a bad argument or allocation failure; -2 when out_cap
 * was too small (*n_out then says how many are needed).
 */
static int orc_trace_core(const int dims[3], double box_len_cm, const double *n_H, const double *x_HI,
                          const double *n_he, int nsrc, const double *pos_cm, const double *ndot,
                          const double *e_ph_eV, const double *sigma_cm2, const int *src_type, int level0,
                          double phi_c, double f_term, int max_level, double *kph, double *gamma, double *budget,
                          uint64_t *counts, uint64_t *hashes, uint64_t *segments, int fc, int src_offset, int n_ages,
                          const double *rlim, size_t n_in, const orc_flight *in, size_t out_cap, orc_flight *out,
                          size_t *n_out, uint64_t root_lo, uint64_t root_hi) {
  if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0 || level0 < 0 || max_level > ORC_MAX_LEVEL ||
      level0 > max_level || !(phi_c > 0) || !(f_term > 0 && f_term < 1) || n_ages < 0 ||
      (n_ages == 0 && n_in > 0))
    return -1;
  const int nt = n_he ? ORC_NTYPES : 1;
  for (int i = 0; src_type && i < nsrc; ++i)
    if (src_type[i] < 0 || src_type[i] >= nt) return -1;
  for (size_t i = 0; i < n_in; ++i)
    if (in[i].src >= (uint32_t)nsrc || in[i].age >= (uint32_t)n_ages || in[i].level > (uint32_t)max_level)
      return -1;
  const size_t ncell = (size_t)dims[0] * dims[1] * dims[2];
  double rsplit[ORC_MAX_LEVEL + 1];
  for (int l = 0; l <= ORC_MAX_LEVEL; ++l) /* Eq. "split": Phi < Phi_c <=> R > R_split */
    rsplit[l] = sqrt((12.0 * ldexp(1.0, 2 * l)) / (4.0 * M_PI * phi_c));

  double *n_abs = (double *)malloc((size_t)nt * ncell * sizeof(double));
  double *s = (double *)malloc((size_t)(nsrc > 0 ? nsrc : 1) * 3 * sizeof(double));
  double *heat = (double *)malloc((size_t)(nsrc > 0 ? nsrc : 1) * sizeof(double));
  if (!n_abs || !s || !heat) { free(n_abs); free(s); free(heat); return -1; }
  for (size_t c = 0; c < ncell; ++c) n_abs[c] = n_H[c] * x_HI[c];
  for (size_t c = 0; nt > 1 && c < 2 * ncell; ++c) n_abs[ncell + c] = n_he[c];
  orc_run R;
  memset(&R, 0, sizeof R);
  R.dims = dims;
  R.ncell = ncell;
  R.n_abs = n_abs;
  R.type = src_type;
  R.dx = box_len_cm / dims[0];
  R.vol = R.dx * R.dx * R.dx;
  R.tau_term = -log(f_term); /* reading R3 */
  R.rsplit = rsplit;
  R.max_level = max_level;
  R.fc = fc;
  R.src_offset = src_offset;
  for (int i = 0; i < nsrc; ++i) {
    for (int a = 0; a < 3; ++a) s[3 * i + a] = pos_cm[3 * i + a] / R.dx;
    heat[i] = (e_ph_eV[i] - orc_e_ion[src_type ? src_type[i] : 0]) * ORC_EV_ERG;
  }
  R.s = s;
  R.sigma_cm2 = sigma_cm2;
  R.heat = heat;
  R.n_ages = n_ages;
  R.rlim = rlim;
  R.kph = kph;
  R.gamma = gamma;
  R.counts = counts;
  R.hashes = hashes;
  R.out = out;
  R.out_cap = out_cap;

  /* Step 2: zero the radiation fields */
  for (size_t c = 0; c < (size_t)nt * ncell; ++c) { kph[c] = 0.0; gamma[c] = 0.0; }
  for (int l = 0; l <= ORC_MAX_LEVEL; ++l) { counts[l] = 0; hashes[l] = 0; }
  orc_ksum emitted = {0, 0}, resumed = {0, 0};

  orc_stack st = {NULL, 0, 0};
  int rc = 0;
  const uint64_t npix0 = 12ULL << (2 * level0);
  for (int src = 0; src < nsrc && rc == 0; ++src) {
    /* Step 1: N_pix packages on the initial level, luminosity spread equally
     * (root packages are numbered src * N_pix + pixel; only those in
     * [root_lo, root_hi) are emitted) */
    const double P0 = ndot[src] / (double)npix0;
    for (uint64_t p = 0; p < npix0; ++p) {
      const uint64_t root = (uint64_t)src * npix0 + (npix0 - 1 - p);
      if (root < root_lo || root >= root_hi) continue;
      orc_pkg pk = {(uint32_t)src, (uint32_t)level0, npix0 - 1 - p, 0.0, P0, 0.0, 0, 0, {0, 0, 0}};
      if (orc_push(&st, pk)) { rc = -1; break; }
      orc_kadd(&emitted, P0);
      counts[level0] += 1;
      hashes[level0] += orc_pkg_hash((uint32_t)(src + src_offset), (uint32_t)level0, npix0 - 1 - p);
    }
    /* Steps 3-5: trace until every package is split, absorbed, gone or halted */
    if (rc == 0) rc = orc_walk(&R, &st);
  }
  /* packages halted by the previous trace continue (R15) */
  for (size_t i = 0; i < n_in && rc == 0; ++i) {
    orc_pkg pk = {in[i].src, in[i].level, in[i].pix, in[i].r, in[i].P, in[i].tau, in[i].age, 1,
                  {in[i].cell[0], in[i].cell[1], in[i].cell[2]}};
    if (orc_push(&st, pk)) { rc = -1; break; }
    orc_kadd(&resumed, in[i].P);
    rc = orc_walk(&R, &st);
  }
  free(st.v);
  free(n_abs);
  free(s);
  free(heat);
  if (rc) return rc;
  budget[0] = orc_kval(&emitted);
  budget[1] = orc_kval(&R.absorbed);
  budget[2] = orc_kval(&R.escaped);
  budget[3] = orc_kval(&resumed);
  budget[4] = orc_kval(&R.halted);
  *segments = R.nseg;
  *n_out = R.n_out;
  return R.n_out > out_cap ? -2 : 0;
}

int orc_trace_mf(const int dims[3], double box_len_cm, const double *n_H, const double *x_HI, const double *n_he,
                 int nsrc, const double *pos_cm, const double *ndot, const double *e_ph_eV, const double *sigma_cm2,
                 const int *src_type, int level0, double phi_c, double f_term, int max_level, double *kph,
                 double *gamma, double *budget, uint64_t *counts, uint64_t *hashes, uint64_t *segments, int fc,
                 int src_offset, int n_ages, const double *rlim, size_t n_in, const orc_flight *in, size_t out_cap,
                 orc_flight *out, size_t *n_out) {
  return orc_trace_core(dims, box_len_cm, n_H, x_HI, n_he, nsrc, pos_cm, ndot, e_ph_eV, sigma_cm2, src_type, level0,
                        phi_c, f_term, max_level, kph, gamma, budget, counts, hashes, segments, fc, src_offset, n_ages,
                        rlim, n_in, in, out_cap, out, n_out, 0, UINT64_MAX);
}

/* orc_trace_roots: the pass of orc_trace (H I photons, infinite speed of
 * light) for the root packages src * 12 * 4^level0 + pixel in
 * [root_first, root_first + root_count) only.  The trace is a sum over root
 * packages, so the outputs of disjoint ranges covering every root add up to
 * the whole pass (k_ph, Gamma, budget, counts, checksums, segments); emitted
 * counts the range's roots only. */
int orc_trace_roots(const int dims[3], double box_len_cm, const double *n_H, const double *x_HI, int nsrc,
                    const double *pos_cm, const double *ndot, const double *e_ph_eV, const double *sigma_cm2,
                    int level0, double phi_c, double f_term, int max_level, double *kph, double *gamma,
                    double *budget, uint64_t *counts, uint64_t *hashes, uint64_t *segments, uint64_t root_first,
                    uint64_t root_count) {
  double b5[5];
  size_t n_out = 0;
  if (root_count > UINT64_MAX - root_first) return -1;
  const int rc = orc_trace_core(dims, box_len_cm, n_H, x_HI, NULL, nsrc, pos_cm, ndot, e_ph_eV, sigma_cm2, NULL,
                                level0, phi_c, f_term, max_level, kph, gamma, b5, counts, hashes, segments, 0, 0, 0,
                                NULL, 0, NULL, 0, NULL, &n_out, root_first, root_first + root_count);
  if (rc == 0) { budget[0] = b5[0]; budget[1] = b5[1]; budget[2] = b5[2]; }
  return rc;
}

/* orc_trace_fsl: the same pass for H I photons only. */
int orc_trace_fsl(const int dims[3], double box_len_cm, const double *n_H, const double *x_HI, int nsrc,
                  const double *pos_cm, const double *ndot, const double *e_ph_eV, const double *sigma_cm2,
                  int level0, double phi_c, double f_term, int max_level, double *kph, double *gamma,
                  double *budget, uint64_t *counts, uint64_t *hashes, uint64_t *segments, int fc, int src_offset,
                  int n_ages, const double *rlim, size_t n_in, const orc_flight *in, size_t out_cap,
                  orc_flight *out, size_t *n_out) {
  return orc_trace_mf(dims, box_len_cm, n_H, x_HI, NULL, nsrc, pos_cm, ndot, e_ph_eV, sigma_cm2, NULL, level0, phi_c,
                      f_term, max_level, kph, gamma, budget, counts, hashes, segments, fc, src_offset, n_ages, rlim,
                      n_in, in, out_cap, out, n_out);
}

/* orc_trace: the same pass with an infinite speed of light (budget[3]:
 * emitted, absorbed, escaped). */
int orc_trace(const int dims[3], double box_len_cm, const double *n_H, const double *x_HI, int nsrc,
              const double *pos_cm, const double *ndot, const double *e_ph_eV,
              const double *sigma_cm2, int level0, double phi_c, double f_term, int max_level,
              double *kph, double *gamma, double *budget, uint64_t *counts, uint64_t *hashes,
              uint64_t *segments, int fc, int src_offset) {
  double b5[5];
  size_t n_out = 0;
  const int rc = orc_trace_fsl(dims, box_len_cm, n_H, x_HI, nsrc, pos_cm, ndot, e_ph_eV, sigma_cm2, level0,
                               phi_c, f_term, max_level, kph, gamma, b5, counts, hashes, segments, fc, src_offset,
                               0, NULL, 0, NULL, 0, NULL, &n_out);
  if (rc == 0) { budget[0] = b5[0]; budget[1] = b5[1]; budget[2] = b5[2]; }
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Chemistry: Eq. "dndt" (readings R6, R7) for every cell.                    */
/*   dx/dt = alpha_B n_H (1 - x)^2 - k_ph x,   x = x_HI,  z = x_HII = 1 - x   */
/* Backward Euler over a substep h, with a = h alpha_B n_H, b = 1 + h k:      */
/*   a x'^2 - (2a + b) x' + (a + x) = 0, physical root x' <= 1, written in    */
/*   the cancellation-free forms                                              */
/*   x' = 2(a + x) / (2a + b + sqrt(D)),  z' = 2(z + hk) / (b + sqrt(D)),     */
/*   D = b^2 + 4a(z + hk).  The smaller of x', z' is kept as computed and the */
/*   other is its complement, so each fraction keeps its relative accuracy.   */
/* ------------------------------------------------------------------------- */
void orc_chem(size_t ncell, const double *n_H, double *x_HI, double *x_HII, const double *kph,
              double dt, int nsub, double alpha_B) {
  const double h = dt / nsub;
  for (size_t c = 0; c < ncell; ++c) {
    double x = x_HI[c], z = x_HII[c];
    const double a = h * alpha_B * n_H[c];
    const double hk = h * kph[c];
    const double b = 1.0 + hk;
    for (int i = 0; i < nsub; ++i) {
      const double D = b * b + 4.0 * a * (z + hk);
      const double sq = sqrt(D);
      const double xn = 2.0 * (a + x) / (2.0 * a + b + sq);
      const double zn = 2.0 * (z + hk) / (b + sq);
      if (xn <= zn) { x = xn; z = 1.0 - xn; }
      else { z = zn; x = 1.0 - zn; }
    }
    x_HI[c] = x;
    x_HII[c] = z;
  }
}
