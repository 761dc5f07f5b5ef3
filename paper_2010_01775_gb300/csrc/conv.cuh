// Convolution launch descriptor and the per-precision forward passes.
#pragma once

#include "pg_internal.cuh"

namespace pgi {

// One convolution layer as an implicit GEMM.  Activations are channel-last;
// `in_cs`/`out_cs` are the channel strides (elements per pixel) and
// `in_co`/`out_co` the first channel used, so a layer can read or write a
// channel slice of a concatenation buffer.  With `ups` set the output pixel
// (y, x) is written to the four pixels (2y + {0,1}, 2x + {0,1}) of a map of
// twice the size (nearest x2 upsampling folded into the store).
struct ConvArgs {
  const void *in;
  int in_cs, in_co, Hin, Win, Cin;
  void *out;
  int out_cs, out_co, Hout, Wout, Cout;
  int k, stride, pad;
  const float *w;     // FP32 weights [K][Cout], K = k*k*Cin
  const float *bias;  // [Cout]
  long M;             // leaves x Hout x Wout
  int act;            // 0 none, 1 ELU, 2 softplus
  int ups;
  int dil;            // tap spacing (dilated convolution); 0 means 1
  // Partial convolution: per output pixel [M] scale k^2 / (valid inputs under
  // the window), 0 where none is valid (output act(0)); null for a plain layer.
  const float *scale;
  // Residual link: added after the activation, same pixel indexing as the
  // output (no upsampling), channel stride res_cs, first channel res_co.
  const void *res;
  int res_cs, res_co;
};

pg_status conv_f32(pg_ctx *ctx, const ConvArgs &a, cudaStream_t st);
pg_status forward_f32(pg_ctx *ctx, const Net *net, const float *x0, void *act, uint32_t ns, int H, int W, float *y,
                      cudaStream_t st);
// Tensor-core (tcgen05) forms.
pg_status tc_prepare(pg_ctx *ctx, Net *net, pg_precision prec);
pg_status forward_tc(pg_ctx *ctx, const Net *net, pg_precision prec, const float *x0, void *act, uint32_t ns,
                     int H, int W, float *y, cudaStream_t st, bool tune = false);
size_t tc_bytes_per_leaf(const Net *net, pg_precision prec, int H, int W);
// BF16 U-Net mixture of experts, one launch per layer over every expert's
// tiles: chunk positions [d_range[e] - pos0, d_range[e+1] - pos0) run expert
// e (ranges padded so that no tile spans two experts); the packed input is
// already assembled at the start of act.
pg_status forward_tc_experts(pg_ctx *ctx, const Net *const *nets, int n_exp, const int *d_range, int pos0, void *act,
                             uint32_t ns, int H, int W, float *y, cudaStream_t st);
int tc_max_experts();

// Masks and partial-convolution scales of the paper-style network (arch 2),
// computed once per chunk from the input mask (the B channel): scale[l] is
// the [ns][Hout][Wout] map of layer l (null for the head).
struct PaperMasks {
  const float *scale[12];
};
size_t paper_mask_floats_per_leaf(int H, int W);
pg_status paper_masks(pg_ctx *ctx, const float *x0, uint32_t ns, int H, int W, float *buf, PaperMasks *pm,
                      cudaStream_t st);

}  // namespace pgi
