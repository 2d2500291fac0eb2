// Work queue of the batched solve: a class of problems of equal structure
// served by several graph branches, each taking the next problem from the
// class's device counter (k_queue_next).
#pragma once

#include "rtg_internal.cuh"

namespace rtg {

struct QueueArgs {
  const SolveDesc* desc;     // the class's problems' descriptors
  InfoDev* info;             // their info records
  unsigned* counter;         // next problem to hand out (zeroed before each launch)
  int n;                     // problems in the class
  int pad;
  SolveDesc* my_desc;        // the branch's descriptor, read by its kernels
  const InfoDev* my_info;    // the branch's info record, written by its epilogue
  int* cur;                  // the branch's current problem (-1: none)
  unsigned long long cond;   // the branch's outer loop condition (cudaGraphConditionalHandle)
  unsigned long long inner;  // the solve's loop condition, set to 1 for a new problem (when use_inner)
  int use_inner;
  int pad2;
};
cudaError_t launch_queue_next(const QueueArgs& q, int done, cudaStream_t s);

}  // namespace rtg
