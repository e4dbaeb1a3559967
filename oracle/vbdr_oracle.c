/*
 * vbdr_oracle.c -- plain, single-threaded CPU oracle of the VBDR method
 * (Xu, "Cardinalities estimation under sliding time window by sharing
 * HyperLogLog Counter", arXiv 1810.13132).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness yardstick of the
 * CUDA library: it shares no code, header, table or constant generator with
 * the library under paper_1810_13132_gb300/, and nothing in the product path
 * may load it.  Only tests/, __graft_entry__.smoke() and the CPU-baseline leg
 * of bench.py use it.
 *
 * Everything is written for clarity, not speed: logical (unpacked) state,
 * one pair at a time, in input order, exactly in the paper's step order.
 *
 *   Sec. 3   Bit distance recorder: DR operations InitDR/SetDR/SlideDR/
 *            IsActiveDR, Alg. 1 EndSliceUpdateBDR, Alg. 2 GetLBP1BDR.
 *   Sec. 4.1 Alg. 3 getPhyIdx, Alg. 4 scanIPpair (VBDR-serial),
 *            Alg. 5 getSumLBP1 followed by the virtual-register-sharing
 *            HyperLogLog estimator the paper cites (vHLL, its ref. TON2017).
 *   Sec. 4.2 bsLBP1 bit string, Alg. 6 EndSliceUpdateBDRGpu, Alg. 7
 *            scanIPpairOnGpu (VBDR-gfast); Alg. 8 BeginSliceUpdateDRV and
 *            Alg. 9 scanIPpairUpdatDRV (VBDR-gsmall); Table 1.
 *
 * Readings of places where the paper is silent or garbled, each with the
 * reason it is taken:
 *   H(x,N,A)  : the paper only says "random hash with seed A mapping x into
 *               [0,N)" (Sec. 4.1).  Read as the SplitMix64 finaliser
 *               (Steele, Lea & Flood 2014):
 *                 H(x,N,A) = (hi32(mix64(x ^ mix64(A))) * N) >> 32.
 *               Seeds: A0 = seed, A1 = mix64(seed + 0x9E3779B97F4A7C15).
 *   LBP1 (rho): leftmost-1 position of bip' << b, counted from 1 as in
 *               HyperLogLog; the all-zero word and positions past the host's
 *               32-b significant bits are capped at 32-b.
 *   DR width  : w = ceil(log2(k+1)) bits, DR_MAX = 2^w - 1 (Sec. 3 gives the
 *               minimum).  SlideDR saturates at DR_MAX (the printed bound
 *               2^k-1 would overflow a w-bit DR).
 *   DRV       : entries 1..R with R = 32 - b_min (entry 0 unused, Alg. 2's
 *               "return 0" is the empty register).
 *   Alg. 1/6  : after the fold nowLBP1 / bsLBP1 is cleared, and a BDR that
 *               received nothing in the slice sets no DR.  Alg. 6's loop is
 *               read as "highest SET bit of bsLBP1 over 32-b bits".
 *   gsmall    : the slice boundary first reads the registers of the window
 *               that just closed (Alg. 2), then runs Alg. 8 for the next
 *               slice; the stored state after a slide is the aged state.
 *   estimator : vHLL,  n = (Z g / (Z - g)) (n_g / g - n_Z / Z),  n_g the HLL
 *               estimate of the host's g virtual registers, n_Z the HLL
 *               estimate of all Z physical registers, each with HLL's
 *               small-range linear counting; clamped at 0.  The harmonic
 *               sums are exact integers S = sum 2^(32 - M).
 *   LogLog /  : Sec. 4.1 notes that the BDR pool can serve PCSA and LogLog
 *   PCSA        counting too.  LogLog (Durand & Flajolet 2003) reads the same
 *               registers (Alg. 5's sum of LBP1 is its statistic):
 *               n_m = alpha_m m 2^(sum M / m), alpha_m =
 *               (Gamma(-1/m) (1 - 2^(1/m)) / ln 2)^(-m).  PCSA (Flajolet &
 *               Martin 1985) keeps a bitmap per BDR: position r is set in the
 *               window iff DR[r] is active, and the BDR's statistic R_j is
 *               the index of its lowest unset position (r - 1 for the first
 *               inactive r, R if all are active); n_m = (m / 0.77351)
 *               2^(sum R_j / m).  Only gsmall records every LBP1 seen (Alg.
 *               9); gfast and serial record a slice maximum, so PCSA reads
 *               gsmall.  Both take the same virtual-sharing noise removal
 *               as vHLL.
 *   mixed g   : the paper gives every host the same g.  For workloads with
 *               mixed g, group_rule 1 assigns host aip  b = b_min + (aip >> 30):
 *               four groups g = 2^b_min .. 2^(b_min+3) selected by the top two
 *               address bits (a workload convention, not a hash).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GFAST 0
#define ORC_GSMALL 1
#define ORC_SERIAL 2

/* ---------------------------------------------------------------- hashing */

/* SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014). */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* One step of the SplitMix64 generator: advances *state, returns output.
 * Exposed only so that the tests can compare with the published
 * known-answer sequence of the generator. */
uint64_t orc_splitmix64_next(uint64_t *state) {
  *state += 0x9e3779b97f4a7c15ULL;
  return orc_mix64(*state);
}

/* H(x, N, A): Sec. 4.1, "random hash function with seed A that maps an
 * integer x to an integer smaller than N".  1 <= N <= 2^32. */
uint64_t orc_H(uint64_t x, uint64_t N, uint64_t A) {
  uint64_t hi32 = orc_mix64(x ^ orc_mix64(A)) >> 32;
  return (hi32 * N) >> 32;
}

/* LB(x, i): Sec. 4.1, the left i bits of the 32-bit word x. */
static uint32_t orc_LB(uint32_t x, uint32_t i) {
  if (i == 0) return 0;
  return x >> (32 - i);
}

/* LBP1 of a 32-bit word, counted from 1 at the most significant bit, as in
 * HyperLogLog (Sec. 3).  Returns 33 for the all-zero word. */
static uint32_t orc_leftmost_one(uint32_t x) {
  uint32_t pos = 1;
  for (int bit = 31; bit >= 0; --bit, ++pos)
    if ((x >> bit) & 1u) return pos;
  return 33;
}

/* ------------------------------------------------------------------ state */

typedef struct {
  int variant;          /* ORC_GFAST / ORC_GSMALL / ORC_SERIAL           */
  uint32_t k;           /* slices per window                             */
  uint64_t Z;           /* physical BDRs in the pool BDRP                */
  uint32_t b_default;   /* log2 g of every host (group_rule 0)           */
  uint32_t b_min;       /* smallest log2 g in use; R = 32 - b_min        */
  uint32_t group_rule;  /* 0: all hosts b_default; 1: four mixed groups  */
  uint64_t A0, A1;      /* hash seeds                                    */
  uint32_t w, dr_max, R;
  uint8_t *DR;          /* [Z][R+1], entry 0 unused                      */
  uint32_t *bs;         /* [Z] bsLBP1 (gfast)                            */
  uint8_t *now;         /* [Z] nowLBP1 (serial)                          */
  uint8_t *reg;         /* [Z] register value of every physical BDR      */
  uint8_t *pcsa;        /* [Z] PCSA statistic of every physical BDR      */
  uint64_t S_Z, V_Z;    /* pool sums of the last slide                   */
  uint64_t L_Z, P_Z;    /* pool sums of registers and PCSA statistics    */
  uint64_t slices_closed;
} orc_t;

static uint32_t orc_dr_width(uint32_t k) {
  uint32_t w = 0;
  while ((1u << w) < k + 1) ++w; /* smallest w with 2^w >= k+1 */
  return w;
}

/* Returns NULL on invalid parameters or allocation failure. */
orc_t *orc_create(int variant, uint32_t k, uint64_t Z, uint32_t b_default,
                  uint32_t b_min, uint32_t group_rule, uint64_t seed) {
  /* Z < 2^32: the exact pool sum sum_j 2^(32 - reg_j) <= Z 2^32 fits 64 bits */
  if (variant < 0 || variant > 2 || k == 0 || Z == 0 || Z >= (1ULL << 32))
    return NULL;
  if (group_rule > 1 || b_min < 1 || b_min > 16) return NULL;
  if (group_rule == 0 && (b_default < b_min || b_default > 16)) return NULL;
  uint32_t b_max = group_rule ? b_min + 3 : b_default;
  if (Z <= (1ULL << b_max)) return NULL; /* Z - g must be positive */
  orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
  if (!o) return NULL;
  o->variant = variant;
  o->k = k;
  o->Z = Z;
  o->b_default = b_default;
  o->b_min = b_min;
  o->group_rule = group_rule;
  o->A0 = seed;
  o->A1 = orc_mix64(seed + 0x9e3779b97f4a7c15ULL);
  o->w = orc_dr_width(k);
  o->dr_max = (1u << o->w) - 1u;
  o->R = 32u - b_min;
  if (o->w > 8) { free(o); return NULL; }
  o->DR = (uint8_t *)malloc((size_t)Z * (o->R + 1));
  o->bs = (uint32_t *)calloc((size_t)Z, sizeof(uint32_t));
  o->now = (uint8_t *)calloc((size_t)Z, 1);
  o->reg = (uint8_t *)calloc((size_t)Z, 1);
  o->pcsa = (uint8_t *)calloc((size_t)Z, 1);
  if (!o->DR || !o->bs || !o->now || !o->reg || !o->pcsa) {
    free(o->DR); free(o->bs); free(o->now); free(o->reg); free(o->pcsa); free(o);
    return NULL;
  }
  /* InitDR on every DR (Sec. 3): value 2^w - 1. */
  memset(o->DR, (int)o->dr_max, (size_t)Z * (o->R + 1));
  return o;
}

void orc_destroy(orc_t *o) {
  if (!o) return;
  free(o->DR); free(o->bs); free(o->now); free(o->reg); free(o->pcsa); free(o);
}

uint32_t orc_dr_max(const orc_t *o) { return o->dr_max; }
uint32_t orc_R(const orc_t *o) { return o->R; }
uint64_t orc_A1(const orc_t *o) { return o->A1; }

/* log2 g of host aip. */
uint32_t orc_host_b(const orc_t *o, uint32_t aip) {
  if (o->group_rule == 0) return o->b_default;
  return o->b_min + (aip >> 30);
}

/* Alg. 3 getPhyIdx. */
uint64_t orc_get_phy_idx(const orc_t *o, uint32_t aip, uint32_t i) {
  uint64_t s1 = orc_H(i, 1ULL << 32, o->A0);
  return orc_H(aip, o->Z, s1);
}

/* The per-pair steps shared by Alg. 4, 7 and 9: hash bip with A1, take the
 * virtual index from its left b bits, shift them out, map (aip, vidx) to a
 * physical BDR and take LBP1 of the shifted word. */
void orc_hash_pair(const orc_t *o, uint32_t aip, uint32_t bip,
                   uint64_t *pidx, uint32_t *rho, uint32_t *vidx) {
  uint32_t b = orc_host_b(o, aip);
  uint32_t bipp = (uint32_t)orc_H(bip, 1ULL << 32, o->A1);
  uint32_t v = orc_LB(bipp, b);
  uint32_t shifted = bipp << b;
  uint32_t r = orc_leftmost_one(shifted);
  if (r > 32 - b) r = 32 - b;
  *vidx = v;
  *rho = r;
  *pidx = orc_get_phy_idx(o, aip, v);
}

/* -------------------------------------------------------------- DR ops */

static uint8_t *orc_drv(orc_t *o, uint64_t j) { return o->DR + j * (o->R + 1); }
static void SetDR(uint8_t *dr) { *dr = 0; }
static void SlideDR(const orc_t *o, uint8_t *dr) { if (*dr < o->dr_max) (*dr)++; }
static int IsActiveDR(const orc_t *o, uint8_t dr) { return dr < o->k; }

/* Alg. 2 GetLBP1BDR: the largest LBP1 whose DR is active, else 0. */
static uint32_t GetLBP1BDR(const orc_t *o, uint64_t j) {
  const uint8_t *drv = o->DR + j * (o->R + 1);
  for (uint32_t lbp1 = o->R; lbp1 >= 1; --lbp1)
    if (IsActiveDR(o, drv[lbp1])) return lbp1;
  return 0;
}

/* PCSA statistic of a BDR's window bitmap (position r set iff DR[r] is
 * active): the index of the lowest unset position, counted from 0. */
static uint32_t PcsaBDR(const orc_t *o, uint64_t j) {
  const uint8_t *drv = o->DR + j * (o->R + 1);
  for (uint32_t r = 1; r <= o->R; ++r)
    if (!IsActiveDR(o, drv[r])) return r - 1;
  return o->R;
}

/* ------------------------------------------------------------ the scan */

/* One time slice of pairs, AoS (aip, bip), in input order.
 *   serial: Alg. 4 first loop   nowLBP1 = max(nowLBP1, LBP1)
 *   gfast : Alg. 7              bsLBP1[LBP1] = 1
 *   gsmall: Alg. 9              SetDR(DRV[LBP1])                      */
void orc_scan(orc_t *o, const uint32_t *pairs, uint64_t n) {
  for (uint64_t p = 0; p < n; ++p) {
    uint64_t pidx;
    uint32_t rho, vidx;
    orc_hash_pair(o, pairs[2 * p], pairs[2 * p + 1], &pidx, &rho, &vidx);
    if (o->variant == ORC_SERIAL) {
      if (rho > o->now[pidx]) o->now[pidx] = (uint8_t)rho;
    } else if (o->variant == ORC_GFAST) {
      o->bs[pidx] |= 1u << (rho - 1); /* bit rho-1 <-> LBP1 value rho */
    } else {
      SetDR(&orc_drv(o, pidx)[rho]);
    }
  }
}

static void orc_pool_sums(orc_t *o) {
  uint64_t S = 0, V = 0, L = 0, P = 0;
  for (uint64_t j = 0; j < o->Z; ++j) {
    S += 1ULL << (32 - o->reg[j]);
    V += (o->reg[j] == 0);
    L += o->reg[j];
    P += o->pcsa[j];
  }
  o->S_Z = S;
  o->V_Z = V;
  o->L_Z = L;
  o->P_Z = P;
}

/* Slice boundary.
 *   serial: Alg. 1 on every BDR (slide all DRs, SetDR(DRV[nowLBP1])).
 *   gfast : Alg. 6 on every BDR (slide all DRs, SetDR at the highest set
 *           bit of bsLBP1), then bsLBP1 is cleared for the next slice.
 *   Both then read every register with Alg. 2.
 *   gsmall: read every register with Alg. 2 (window closed), then Alg. 8
 *           (slide all DRs) for the next slice.                       */
void orc_slide(orc_t *o) {
  for (uint64_t j = 0; j < o->Z; ++j) {
    uint8_t *drv = orc_drv(o, j);
    if (o->variant == ORC_GSMALL) {
      o->reg[j] = (uint8_t)GetLBP1BDR(o, j);
      o->pcsa[j] = (uint8_t)PcsaBDR(o, j);
      for (uint32_t r = 1; r <= o->R; ++r) SlideDR(o, &drv[r]);
      continue;
    }
    for (uint32_t r = 1; r <= o->R; ++r) SlideDR(o, &drv[r]);
    uint32_t lbp1 = 0;
    if (o->variant == ORC_SERIAL) {
      lbp1 = o->now[j];
      o->now[j] = 0;
    } else {
      for (uint32_t i = 0; i < o->R; ++i)
        if ((o->bs[j] >> i) & 1u) lbp1 = i + 1; /* highest set bit */
      o->bs[j] = 0;
    }
    if (lbp1 > 0) SetDR(&drv[lbp1]);
    o->reg[j] = (uint8_t)GetLBP1BDR(o, j);
    /* a slice maximum is no bitmap: no PCSA statistic outside gsmall */
  }
  orc_pool_sums(o);
  o->slices_closed++;
}

/* ------------------------------------------------------- the estimator */

/* HyperLogLog bias constant alpha_m (Flajolet et al. 2007). */
double orc_hll_alpha(double m) {
  if (m == 16) return 0.673;
  if (m == 32) return 0.697;
  if (m == 64) return 0.709;
  return 0.7213 / (1.0 + 1.079 / m);
}

/* HLL raw estimate from m registers with harmonic sum sum_j 2^-M_j =
 * S * 2^-32 and V empty registers, with small-range linear counting. */
double orc_hll(double m, uint64_t S, uint64_t V) {
  double harmonic = ldexp((double)S, -32);
  double E = orc_hll_alpha(m) * m * m / harmonic;
  if (E <= 2.5 * m && V > 0) E = m * log(m / (double)V);
  return E;
}

/* vHLL with virtual register sharing. */
/* The virtual-sharing noise removal of vHLL, n = Z g / (Z - g) (n_g / g -
 * n_Z / Z) clamped at 0, for any estimator of the host's registers (n_g)
 * and of the pool (n_Z). */
static double orc_denoise(double Z, double g, double n_g, double n_Z) {
  double n = (Z * g / (Z - g)) * (n_g / g - n_Z / Z);
  return n > 0.0 ? n : 0.0;
}

double orc_vhll(double Z, double g, uint64_t S, uint64_t V, uint64_t S_Z,
                uint64_t V_Z) {
  return orc_denoise(Z, g, orc_hll(g, S, V), orc_hll(Z, S_Z, V_Z));
}

/* LogLog bias constant (Durand & Flajolet 2003):
 *   alpha_m = (Gamma(-1/m) (1 - 2^(1/m)) / ln 2)^(-m),
 * with 1 - 2^(1/m) = -expm1(ln 2 / m) to keep its digits for large m. */
double orc_loglog_alpha(double m) {
  double base = tgamma(-1.0 / m) * -expm1(log(2.0) / m) / log(2.0);
  return pow(base, -m);
}

/* LogLog estimate of m registers whose values sum to L. */
double orc_loglog(double m, uint64_t L) {
  return orc_loglog_alpha(m) * m * exp2((double)L / m);
}

/* PCSA estimate of m bitmaps whose statistics sum to P (Flajolet & Martin
 * 1985, phi = 0.77351). */
double orc_pcsa(double m, uint64_t P) {
  return m / 0.77351 * exp2((double)P / m);
}

/* Alg. 5 getSumLBP1 generalised: visits the host's g virtual registers
 * (Alg. 3 then Alg. 2, read here from reg[] which holds Alg. 2 of every
 * BDR at the last slide) and collects the exact harmonic sum, the number of
 * empty registers, the plain LBP1 sum and a 64-bin register histogram. */
void orc_host_registers(const orc_t *o, uint32_t aip, uint64_t *S,
                        uint64_t *V, uint64_t *sum_lbp1, uint32_t *hist64) {
  uint32_t b = orc_host_b(o, aip);
  uint32_t g = 1u << b;
  uint64_t s = 0, v = 0, l = 0;
  if (hist64) memset(hist64, 0, 64 * sizeof(uint32_t));
  for (uint32_t i = 0; i < g; ++i) {
    uint32_t M = o->reg[orc_get_phy_idx(o, aip, i)];
    s += 1ULL << (32 - M);
    v += (M == 0);
    l += M;
    if (hist64) hist64[M]++;
  }
  *S = s;
  *V = v;
  if (sum_lbp1) *sum_lbp1 = l;
}

/* Per-host feature vector of the learned correction (not part of the
 * paper; its definition is shared by specification with the library):
 *   x[v]  = #{virtual registers with value v} / g,   v = 0..63
 *   x[64] = b / 16
 *   x[65] = ln(1 + n_plain) / 16      (the vHLL estimate)
 *   x[66] = ln(1 + n_g) / 16          (the host's HLL estimate, noise kept)
 *   x[67] = ln(1 + n_Z / Z)           (pool load per register)
 *   x[68] = V_Z / Z                   (pool empty fraction)
 *   x[69] = V / g                     (host empty fraction)
 *   x[70..79] = 0
 * X is [n][80]; n_plain[h] receives the vHLL estimate. */
int orc_features(const orc_t *o, const uint32_t *aips, uint64_t n, double *X,
                 double *n_plain) {
  if (o->slices_closed == 0) return -1;
  const double Z = (double)o->Z;
  const double n_Z = orc_hll(Z, o->S_Z, o->V_Z);
  for (uint64_t h = 0; h < n; ++h) {
    uint64_t S, V;
    uint32_t hist[64];
    orc_host_registers(o, aips[h], &S, &V, NULL, hist);
    uint32_t b = orc_host_b(o, aips[h]);
    double g = (double)(1u << b);
    double n_g = orc_hll(g, S, V);
    double est = orc_vhll(Z, g, S, V, o->S_Z, o->V_Z);
    double *x = X + h * 80;
    for (int v = 0; v < 64; ++v) x[v] = hist[v] / g;
    x[64] = b / 16.0;
    x[65] = log1p(est) / 16.0;
    x[66] = log1p(n_g) / 16.0;
    x[67] = log1p(n_Z / Z);
    x[68] = (double)o->V_Z / Z;
    x[69] = (double)V / g;
    for (int v = 70; v < 80; ++v) x[v] = 0.0;
    n_plain[h] = est;
  }
  return 0;
}

/* Estimates of n hosts, FP64.  Returns -1 before the first slide. */
int orc_estimate(const orc_t *o, const uint32_t *aips, uint64_t n,
                 double *out) {
  if (o->slices_closed == 0) return -1;
  for (uint64_t h = 0; h < n; ++h) {
    uint64_t S, V;
    orc_host_registers(o, aips[h], &S, &V, NULL, NULL);
    double g = (double)(1u << orc_host_b(o, aips[h]));
    out[h] = orc_vhll((double)o->Z, g, S, V, o->S_Z, o->V_Z);
  }
  return 0;
}

/* Estimates with the LogLog (which = 1) or PCSA (which = 2) statistic of
 * the host's g virtual BDRs, FP64.  Alg. 5's getSumLBP1 is the LogLog sum.
 * Returns -1 before the first slide, -2 for PCSA on a layout other than
 * gsmall. */
int orc_estimate_alt(const orc_t *o, int which, const uint32_t *aips, uint64_t n,
                     double *out) {
  if (o->slices_closed == 0) return -1;
  if (which == 2 && o->variant != ORC_GSMALL) return -2;
  const double Z = (double)o->Z;
  const double n_Z = which == 1 ? orc_loglog(Z, o->L_Z) : orc_pcsa(Z, o->P_Z);
  for (uint64_t h = 0; h < n; ++h) {
    uint32_t b = orc_host_b(o, aips[h]);
    uint32_t g = 1u << b;
    uint64_t sum = 0;
    for (uint32_t i = 0; i < g; ++i) {
      uint64_t j = orc_get_phy_idx(o, aips[h], i);
      sum += which == 1 ? o->reg[j] : o->pcsa[j];
    }
    double n_g = which == 1 ? orc_loglog((double)g, sum) : orc_pcsa((double)g, sum);
    out[h] = orc_denoise(Z, (double)g, n_g, n_Z);
  }
  return 0;
}

/* ---------------------------------------------------------- inspection */

/* Logical state: DR as [Z][R] (entries 1..R), bs [Z], reg [Z]; any output
 * pointer may be NULL. */
void orc_get_state(const orc_t *o, uint8_t *dr_out, uint32_t *bs_out,
                   uint8_t *reg_out, uint8_t *now_out) {
  for (uint64_t j = 0; j < o->Z; ++j) {
    if (dr_out)
      memcpy(dr_out + j * o->R, o->DR + j * (o->R + 1) + 1, o->R);
    if (bs_out) bs_out[j] = o->bs[j];
    if (reg_out) reg_out[j] = o->reg[j];
    if (now_out) now_out[j] = o->now[j];
  }
}

/* Overwrite the logical DRV ([Z][R], entries 1..R) and bsLBP1 ([Z]); either
 * pointer may be NULL.  Used to install a state merged from several
 * replicas that each scanned part of a slice. */
void orc_set_state(orc_t *o, const uint8_t *dr_in, const uint32_t *bs_in) {
  for (uint64_t j = 0; j < o->Z; ++j) {
    if (dr_in) memcpy(o->DR + j * (o->R + 1) + 1, dr_in + j * o->R, o->R);
    if (bs_in) o->bs[j] = bs_in[j];
  }
}

/* Overwrite the register array and recompute the pool sums: used to put a
 * register-level synthetic state (one whose scan would be too long to run)
 * under the estimator. */
void orc_set_registers(orc_t *o, const uint8_t *reg_in) {
  memcpy(o->reg, reg_in, (size_t)o->Z);
  orc_pool_sums(o);
  if (o->slices_closed == 0) o->slices_closed = 1;
}

/* Register-level synthetic state, for workloads too large to scan: every
 * physical register becomes the largest of the virtual register values that
 * Alg. 3 maps onto it (host aips[h]'s virtual index i goes to BDR
 * getPhyIdx(aips[h], i)); registers no virtual register maps to are 0.
 * vregs[offsets[h] + i], i < g(aips[h]), is host h's i-th value. */
void orc_load_virtual_registers(orc_t *o, const uint32_t *aips, const uint64_t *offsets,
                                uint64_t n, const uint8_t *vregs) {
  memset(o->reg, 0, (size_t)o->Z);
  for (uint64_t h = 0; h < n; ++h) {
    uint32_t g = 1u << orc_host_b(o, aips[h]);
    for (uint32_t i = 0; i < g; ++i) {
      uint64_t j = orc_get_phy_idx(o, aips[h], i);
      uint8_t v = vregs[offsets[h] + i];
      if (v > o->reg[j]) o->reg[j] = v;
    }
  }
  orc_pool_sums(o);
  if (o->slices_closed == 0) o->slices_closed = 1;
}

void orc_pool_sums_get(const orc_t *o, uint64_t *S_Z, uint64_t *V_Z) {
  *S_Z = o->S_Z;
  *V_Z = o->V_Z;
}

/* Pool sums of the registers (LogLog) and PCSA statistics. */
void orc_pool_sums_alt(const orc_t *o, uint64_t *L_Z, uint64_t *P_Z) {
  *L_Z = o->L_Z;
  *P_Z = o->P_Z;
}

/* PCSA statistic of every BDR at the last slide. */
void orc_get_pcsa(const orc_t *o, uint8_t *out) { memcpy(out, o->pcsa, (size_t)o->Z); }

/* Table 1: bits of one BDR per variant, with log2(n/g) read as R DRs and
 * log2(k+1) as the DR width w.  serial stores nowLBP1 in
 * ceil(log2(R+1)) bits, gfast stores bsLBP1 in R bits. */
uint32_t orc_table1_bits(const orc_t *o, int variant) {
  uint32_t drv = o->R * o->w;
  if (variant == ORC_GSMALL) return drv;
  if (variant == ORC_GFAST) return o->R + drv;
  uint32_t nb = 0;
  while ((1u << nb) < o->R + 1) ++nb;
  return nb + drv;
}
