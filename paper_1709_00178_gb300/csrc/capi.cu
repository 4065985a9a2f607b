// C ABI entry points of the single-stripe coding path, the one-shot batched calls and the device
// status word.
#include <cuda_runtime.h>

#include "pyrit_internal.h"

using namespace pyrit;

namespace {

// Codes one job: the staged kernel when P and every pointer allow 16-byte bulk copies, else the
// plain-load kernel. The staged kernel is the generated network of the job's mask table when one
// is compiled (a missing one is queued under PYRIT_JIT_ASYNC), else the generic one. Under the
// parity transform, or for a field the generic kernels are not built for, only a generated
// network codes the job: it is compiled in the call if missing, and anything else is
// PYRIT_E_UNSUPPORTED. The job travels in the kernel's parameters: no coding state is allocated.
int run_job(const pyrit_plan_s* plan, const JobDesc& job, cudaStream_t stream) {
  if (job.nout == 0) return PYRIT_OK;
  const int n = plan->n;
  const bool parity = network_only(plan);
  if (job_is_staged(job)) {
    TileShape sh;
    const Variant* net = net_variant(net_spec(n, job, 0, 0, 0, 0, plan->transform, plan_net_g(plan)), parity);
    if (net)
      shape_for_variant(net, job.nout, ShapeHint(), &sh);
    else if (parity)
      return PYRIT_E_UNSUPPORTED;
    else if (!choose_shape(n, job.nout, ShapeHint(), &sh))
      return PYRIT_E_UNSUPPORTED_FIELD;
    const uint32_t tpj = tiles_for(job.P, sh);
    return launch_staged(sh, &job, nullptr, nullptr, tpj, tpj, stream);
  }
  if (parity) return PYRIT_E_UNSUPPORTED;
  return launch_plain(n, job, stream);
}

// Codes a stripe's jobs in order on the stream (one per group of up to kMaxOut outputs; they read
// the same sources). Under the parity transform every job must be able to run on a network
// before the first is launched.
int run_jobs(const pyrit_plan_s* plan, const JobDesc* jobs, int nj, cudaStream_t stream) {
  if (network_only(plan))
    for (int i = 0; i < nj; ++i)
      if (!job_is_staged(jobs[i])) return PYRIT_E_UNSUPPORTED;
  for (int i = 0; i < nj; ++i) {
    const int rc = run_job(plan, jobs[i], stream);
    if (rc != PYRIT_OK) return rc;
  }
  return PYRIT_OK;
}

}  // namespace

extern "C" {

int pyrit_encode(pyrit_plan_t plan, const void* const* data, void* const* parity, size_t P, pyrit_stream_t stream) {
  if (!plan || !data || (plan->m > 0 && !parity) || P == 0 || P > (1ull << 40)) return PYRIT_E_INVALID_ARG;
  for (int j = 0; j < plan->k; ++j)
    if (!data[j]) return PYRIT_E_INVALID_ARG;
  for (int i = 0; i < plan->m; ++i)
    if (!parity[i]) return PYRIT_E_INVALID_ARG;
  if (plan->m == 0) return PYRIT_OK;
  JobDesc jobs[kMaxJobs];
  const int nj = make_encode_jobs(plan, data, parity, P, jobs);
  return run_jobs(plan, jobs, nj, reinterpret_cast<cudaStream_t>(stream));
}

int pyrit_decode(pyrit_plan_t plan, void* const* blocks, uint64_t erasures, size_t P, pyrit_stream_t stream) {
  if (!plan || !blocks || P == 0 || P > (1ull << 40)) return PYRIT_E_INVALID_ARG;
  const int nb = plan->k + plan->m;
  for (int b = 0; b < nb; ++b)
    if (!blocks[b]) return PYRIT_E_INVALID_ARG;
  DecodeEntry e;
  const int rc = plan_decode_entry(plan, erasures, &e);
  if (rc != PYRIT_OK) return rc;
  if (e.ne == 0) return PYRIT_OK;
  JobDesc jobs[kMaxJobs];
  const int nj = make_decode_jobs(plan, e, blocks, P, jobs);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The plan's syndrome-decode network serves every erasure pattern: used once compiled (compiled
  // in the call under the parity transform, which has no generic kernel). It exists for m <= 8,
  // where the decode is one job.
  if (e.syn_ok && nj == 1 && job_is_staged(jobs[0])) {
    const bool block = network_only(plan);
    JobDesc sj;
    make_syndrome_job(plan, e, blocks, P, &sj);
    // the network's all-rows body when this pattern needs every parity row
    const int allrows = sj.mask[kSyndromeNeedRow][0] == (1u << plan->m) - 1u ? 1 : 0;
    if (const Variant* net = net_variant(net_spec_syndrome(plan, 0, 0, 0, allrows), block)) {
      TileShape sh;
      shape_for_variant(net, plan->m, ShapeHint(), &sh);
      const uint32_t tpj = tiles_for(P, sh);
      return launch_staged(sh, &sj, nullptr, nullptr, tpj, tpj, st);
    }
  }
  return run_jobs(plan, jobs, nj, st);
}

}  // extern "C"

namespace {

// A batch of stripes that all carry `op`, made, run once on `stream`, waited for and freed.
int one_shot_batch(const pyrit_stripe_t* stripes, int count, int op, pyrit_stream_t stream) {
  if (count < 0 || (count > 0 && !stripes)) return PYRIT_E_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (stripes[i].op != op) return PYRIT_E_INVALID_ARG;
  if (count == 0) return PYRIT_OK;
  pyrit_batch_t b = nullptr;
  int rc = pyrit_batch_create(stripes, count, nullptr, &b);
  if (rc != PYRIT_OK) return rc;
  rc = pyrit_batch_run(b, stream, 0);
  // the batch's tables must outlive its launches
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess && rc == PYRIT_OK) rc = PYRIT_E_CUDA;
  pyrit_batch_destroy(b);
  return rc;
}

}  // namespace

extern "C" {

int pyrit_encode_batch(const pyrit_stripe_t* stripes, int count, pyrit_stream_t stream) {
  return one_shot_batch(stripes, count, PYRIT_OP_ENCODE, stream);
}

int pyrit_decode_batch(const pyrit_stripe_t* stripes, int count, pyrit_stream_t stream) {
  return one_shot_batch(stripes, count, PYRIT_OP_DECODE, stream);
}

int pyrit_device_status(int* code_out, int* where_out) {
  if (!code_out) return PYRIT_E_INVALID_ARG;
  int* w = device_error_word();
  if (!w) return PYRIT_E_CUDA;
  int h[2] = {0, 0};
  if (cudaDeviceSynchronize() != cudaSuccess) return PYRIT_E_CUDA;
  if (cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return PYRIT_E_CUDA;
  if (cudaMemset(w, 0, sizeof(h)) != cudaSuccess) return PYRIT_E_CUDA;
  *code_out = h[0];
  if (where_out) *where_out = h[1];
  return PYRIT_OK;
}

}  // extern "C"
