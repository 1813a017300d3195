// Two scattering models written against the four-function interface of
// sidm_model.cuh (Sec. 4.6), as a host code would write them, compiled by
// tests/test_gpu_model_interface.py into a shared library of its own.
//
// UserElastic restates the elastic isotropic scatter of Sec. 4.1 with its own
// code: a direction uniform on the sphere by Marsaglia's (1972) rejection
// from the pair's random streams 1, 2, ..., and the centre-of-momentum kick
// v_com = ((m_a v_a) + (m_b v_b)) / M, g = |v_a - v_b|,
// v_a' = v_com + ((m_b g) / M) e, v_b' = v_com - ((m_a g) / M) e,
// every operation rounded once in that order (IEEE intrinsics, so no
// contraction whatever the compiler flags).
// CountingElastic adds per-particle state the library knows nothing of: a
// count of the scatters of each particle, carried through get_state,
// scatter, overwrite_state and set_state.
#include "sidm_model.cuh"

namespace {

using sidm_model::PairInfo;

struct UserElastic {
  struct State {
    double v[3];
    double m;
  };
  struct Particles {
    double* vel;
    const double* mass;
  };

  __device__ State get_state(const Particles& P, int32_t i) const {
    State s;
    for (int k = 0; k < 3; ++k) s.v[k] = P.vel[3 * (int64_t)i + k];
    s.m = P.mass[i];
    return s;
  }
  __device__ void set_state(const Particles& P, int32_t i, const State& s) const {
    for (int k = 0; k < 3; ++k) P.vel[3 * (int64_t)i + k] = s.v[k];
  }
  __device__ static void unit_vector(const PairInfo& p, double e[3]) {
    e[0] = 0.0;
    e[1] = 0.0;
    e[2] = 1.0;
    for (uint32_t t = 1; t <= 64; ++t) {
      const uint4 w = p.words(t);
      const double x1 = __dsub_rn(__dmul_rn(2.0, sidm_model::unit53(w.x, w.y)), 1.0);
      const double x2 = __dsub_rn(__dmul_rn(2.0, sidm_model::unit53(w.z, w.w)), 1.0);
      const double s = __dadd_rn(__dmul_rn(x1, x1), __dmul_rn(x2, x2));
      if (s > 0.0 && s < 1.0) {
        const double q = __dmul_rn(2.0, __dsqrt_rn(__dsub_rn(1.0, s)));
        e[0] = __dmul_rn(x1, q);
        e[1] = __dmul_rn(x2, q);
        e[2] = __dsub_rn(1.0, __dmul_rn(2.0, s));
        return;
      }
    }
    atomicAdd(p.warnings, 1u);
  }
  __device__ void scatter(State& a, State& b, const PairInfo& p) const {
    double e[3];
    unit_vector(p, e);
    const double M = __dadd_rn(a.m, b.m);
    double vc[3], d[3];
    for (int k = 0; k < 3; ++k) {
      vc[k] = __ddiv_rn(__dadd_rn(__dmul_rn(a.m, a.v[k]), __dmul_rn(b.m, b.v[k])), M);
      d[k] = __dsub_rn(a.v[k], b.v[k]);
    }
    const double g = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                          __dmul_rn(d[2], d[2])));
    const double fa = __ddiv_rn(__dmul_rn(b.m, g), M), fb = __ddiv_rn(__dmul_rn(a.m, g), M);
    for (int k = 0; k < 3; ++k) {
      a.v[k] = __dadd_rn(vc[k], __dmul_rn(fa, e[k]));
      b.v[k] = __dsub_rn(vc[k], __dmul_rn(fb, e[k]));
    }
  }
  __device__ State overwrite_state(const State&, const State& out) const { return out; }
};

struct CountingElastic {
  UserElastic kick;
  struct State {
    UserElastic::State s;
    int count;
  };
  struct Particles {
    UserElastic::Particles p;
    int32_t* count;
  };
  __device__ State get_state(const Particles& P, int32_t i) const {
    return State{kick.get_state(P.p, i), P.count[i]};
  }
  __device__ void set_state(const Particles& P, int32_t i, const State& s) const {
    kick.set_state(P.p, i, s.s);
    P.count[i] = s.count;
  }
  __device__ void scatter(State& a, State& b, const PairInfo& p) const {
    kick.scatter(a.s, b.s, p);
    a.count += 1;
    b.count += 1;
  }
  __device__ State overwrite_state(const State&, const State& out) const { return out; }
};

}  // namespace

extern "C" {

size_t ext_scratch_bytes(int64_t n, int64_t n_pairs) {
  return sidm_model::apply_pairs_scratch_bytes(n, n_pairs);
}

int ext_apply_elastic(const sidm_pair* pairs, int64_t n_pairs, double* vel, const double* mass,
                      int64_t n, uint64_t seed, uint64_t step, void* scratch, size_t bytes,
                      void* stream) {
  return sidm_model::apply_pairs(UserElastic{}, UserElastic::Particles{vel, mass}, pairs, n_pairs,
                                 n, seed, step, scratch, bytes, (cudaStream_t)stream);
}

int ext_apply_counting(const sidm_pair* pairs, int64_t n_pairs, double* vel, const double* mass,
                       int32_t* count, int64_t n, uint64_t seed, uint64_t step, void* scratch,
                       size_t bytes, void* stream) {
  const CountingElastic::Particles P{UserElastic::Particles{vel, mass}, count};
  return sidm_model::apply_pairs(CountingElastic{}, P, pairs, n_pairs, n, seed, step, scratch,
                                 bytes, (cudaStream_t)stream);
}

int ext_apply_builtin(const sidm_pair* pairs, int64_t n_pairs, double* vel, const double* mass,
                      int64_t n, uint64_t seed, uint64_t step, double eps, void* scratch,
                      size_t bytes, void* stream) {
  sidm_model::IsotropicKick m;
  m.eps = eps;
  return sidm_model::apply_pairs(m, sidm_model::IsotropicKick::Particles{vel, mass}, pairs,
                                 n_pairs, n, seed, step, scratch, bytes, (cudaStream_t)stream);
}

}  // extern "C"
