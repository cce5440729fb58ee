// The launch sequence of one decode call (interleave, iterations of the
// chosen schedule, syndrome checks, de-interleave), templated on the message
// storage type and slab width.  Included by decode_f16.cu and decode_f32.cu,
// which compile the half and float kernels as separate translation units.
#pragma once

#include "kernels.cuh"

namespace {

// Launch the full decode sequence on device buffers.
template <typename MsgT, int W>
int run_decode(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syn,
               int32_t batch, int32_t iters, bool et, uint8_t *bits, float *post,
               uint8_t *conv_out, int32_t *iters_out, cudaStream_t st, bool out_dev) {
    const mld::HostGraph &h = d->g->h;
    const mld_graph *g = d->g;
    const int slabs = (batch + W - 1) / W;
    constexpr int TPC = W / kK;
    constexpr int DW = (W + 31) / 32;
    const size_t rbytes = static_cast<size_t>(slabs) * h.e_core * W * sizeof(MsgT);
    if (rbytes) MLD_CUDA(cudaMemsetAsync(d->r, 0, rbytes, st));
    MLD_CUDA(cudaMemsetAsync(d->done, 0, sizeof(uint32_t) * slabs * DW, st));

    // Posterior accumulation: iteration l reads the posteriors of l-1 from
    // one of three buffers and adds its messages into the buffer of l,
    // which starts at L_ch; the rotation ends on d->Lv.
    const bool acc_mode = d->vn_update == MLD_VN_ACCUMULATE && !et && iters > 0 && d->Lv2 && d->Lv3;
    float *const accbuf[3] = {d->Lv, d->Lv2, d->Lv3};
    auto acc_of = [&](int32_t l) { return accbuf[(iters - l) % 3]; };

    d->sample_now = true;
    InArgs ia{in, sigma, g->unit, h.n_vn, h.n_core, h.n_deg1, batch, d->lmax, d->scale_in, d->lmax_i, d->amin_i,
              d->lch, acc_mode ? acc_of(0) : d->Lv, d->lch1, d->post1, d->phi1};
    if (h.n_vn > 0) {
        int s = timed_launch(d, kClsLayout, st, "k_interleave_in", [&] {
            k_interleave_in<W, DecodeFit<MsgT>::value><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(ia);
        });
        if (s != MLD_OK) return s;
    }
    if (h.n_cn > 0) {
        int s = timed_launch(d, kClsLayout, st, "k_syndrome_in", [&] {
            k_syndrome_in<W><<<dim3((h.n_cn + 31) / 32, slabs), kBlock, 0, st>>>(syn, g->cint, h.n_cn, batch,
                                                                                d->sbits);
        });
        if (s != MLD_OK) return s;
    }

    // degree-1 decisions: two buffers, written by iterations of each parity
    // (a codeword's output is read from the one of its last iteration)
    const size_t h1 = static_cast<size_t>(slabs) * h.n_deg1 * (W / 8);
    auto hb1_of = [&](int32_t l) { return d->hb1 + static_cast<size_t>(l & 1) * h1; };
    CnArgs ca{g->cptr, g->col, g->dptr, h.n_cn, h.n_core, h.n_deg1, h.e_core,
              d->r, d->Lv, d->lch1, d->phi1, d->post1, d->hb1, d->sbits, d->done,
              d->lmax_i, d->amin_i, 0, et ? 1 : 0, 0, batch, d->hb1, d->fail};
    ca.status = d->status;
    ca.stall_test = d->stall_test;
    // early termination without soft output: degree-1 decisions only, and
    // the syndrome of iteration l-1 formed inside check pass l (every check
    // in a register class; otherwise a separate syndrome check per iteration)
    ca.rule = d->check_rule == MLD_CHECK_MIN_SUM ? kRuleMinSum : kRuleSumProduct;
    ca.ms_off = d->ms_off_i;
    // (the decision-only form is a sum-product property)
    const bool hard1 = et && !post && d->check_rule == MLD_CHECK_SUM_PRODUCT;
    // the fused syndrome check is for the host-driven loop (decoder views
    // without a capture stream); otherwise the device loop runs the iterations
    const bool fused = hard1 && g->fusable && !d->cap;
    VnArgs va{g->vptr, g->vedge, h.n_core, h.e_core, d->r, d->lch, d->Lv, d->hb_core, d->done, 0, et ? 1 : 0};
    SynArgs sa{g->cptr, g->col, g->dptr, h.n_cn, h.n_core, h.n_deg1, d->sbits, d->hb_core, d->hb1,
               d->fail, d->done, et ? 1 : 0, batch};
    // check-update launches, one per check class (built with the graph)
    const int wi = W == 8 ? 0 : (W == 16 ? 1 : (W == 32 ? 2 : 3));
    const std::vector<ClassLaunch> &launches = g->launches[wi];
    // with a side stream and several classes, the largest runs on `st`
    int big = -1;
    if (d->side && launches.size() > 1) {
        big = 0;
        for (size_t i = 1; i < launches.size(); ++i)
            if (static_cast<int64_t>(launches[i].blocks) * launches[i].deg >
                static_cast<int64_t>(launches[big].blocks) * launches[big].deg)
                big = static_cast<int>(i);
    }
    const dim3 vn_grid(grid_x(static_cast<int64_t>(h.n_core) * TPC), slabs);
    int sm_count = 152;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, d->device);
    const dim3 syn_grid(syndrome_blocks(h.n_cn, sm_count), slabs);
    const int cap_blocks = sm_count * 16;  // two waves of 8 blocks per SM
    // staged check updates: one wave of kStagedBlocksPerSm blocks per SM
    const int staged_cap = d->staging != MLD_STAGE_DIRECT ? sm_count * kStagedBlocksPerSm : 0;
    const int lane_blocks = (batch + 127) / 128;
    const int64_t acc_n4 = static_cast<int64_t>(slabs) * h.n_core * W / 4;
    const int copy_blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((acc_n4 + kBlock - 1) / kBlock,
                                                                                     sm_count * 8)));

    auto syndrome_round = [&](int32_t l, bool et_mode) -> int {
        MLD_CUDA(cudaMemsetAsync(d->fail, 0, sizeof(uint32_t) * slabs * DW, st));
        if (h.n_cn > 0) {
            sa.et = et_mode ? 1 : 0;
            sa.hb1 = hb1_of(l);
            int s = timed_launch(d, kClsSyn, st, "k_syndrome_check", [&] {
                k_syndrome_check<W><<<syn_grid, kBlock, 0, st>>>(sa);
            });
            if (s != MLD_OK) return s;
        }
        return timed_launch(d, kClsSyn, st, "k_lane_update", [&] {
            k_lane_update<W><<<lane_blocks, 128, 0, st>>>(d->done, d->fail, d->iters, d->conv, batch, l,
                                                           et_mode ? 1 : 0);
        });
    };

    if (iters == 0) {
        if (h.n_core > 0) {
            int s = timed_launch(d, kClsLayout, st, "k_hard_bits", [&] {
                k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(h.n_core) * (W / 8)), slabs), kBlock, 0, st>>>(
                    d->Lv, h.n_core, d->hb_core);
            });
            if (s != MLD_OK) return s;
        }
        if (h.n_deg1 > 0) {
            int s = timed_launch(d, kClsLayout, st, "k_hard_bits", [&] {
                k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(h.n_deg1) * (W / 8)), slabs), kBlock, 0, st>>>(
                    d->post1, h.n_deg1, d->hb1);
            });
            if (s != MLD_OK) return s;
        }
        int s = syndrome_round(0, false);
        if (s != MLD_OK) return s;
    }
    // Early termination with the iterations run by the device (a conditional
    // CUDA-graph loop, see k_loop_cond), so no launch follows the iteration at
    // which the last codeword stops.  Decoder views without a capture stream
    // (mld_decode_noalloc) keep the host loop.
    const bool dev_loop = et && iters > 0 && d->cap && d->lctr && (d->schedule == MLD_SCHED_LAYERED || !fused);
    if (dev_loop) {
        // one early-terminated iteration of parity `parity` (l odd: 1), whose
        // number is lctr[0] + off, enqueued on stream s
        auto enqueue_half = [&](int parity, int off, cudaStream_t s) -> int {
            CnArgs c2 = ca;
            c2.final_pass = 1;
            c2.fuse = 0;
            c2.hb1 = d->hb1 + static_cast<size_t>(parity) * h1;
            if (d->schedule == MLD_SCHED_LAYERED) {
                CnArgs la = c2;
                la.col = g->lcol;
                for (const mld::LayerLaunch &ll : g->layer_launches) {
                    const mld::CheckClass &k = h.classes[ll.cls];
                    la.cptr = g->leptr + ll.p0;
                    const int blocks = std::max(1, std::min(grid_x(static_cast<int64_t>(ll.count) * TPC),
                                                            sm_count * kLayeredBlocksPerSm));
                    ClassLaunch cl{k.c0, ll.count, k.dc, k.dc + k.dd, ll.e0, k.s0, blocks};
                    launch_layered<MsgT, W>(la, cl, g->lchk + ll.p0, slabs, s, hard1);
                }
                MLD_LAUNCHED("k_check_layered");
                if (h.n_core > 0) {
                    k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(h.n_core) * (W / 8)), slabs), kBlock, 0, s>>>(
                        d->Lv, h.n_core, d->hb_core);
                    MLD_LAUNCHED("k_hard_bits");
                }
            } else {
                if (big < 0) {
                    for (const ClassLaunch &cl : launches) launch_check_class<MsgT, W>(c2, cl, slabs, s, cap_blocks, hard1, staged_cap, d->staging);
                } else {
                    MLD_CUDA(cudaEventRecord(d->ev_fork, s));
                    MLD_CUDA(cudaStreamWaitEvent(d->side, d->ev_fork, 0));
                    launch_check_class<MsgT, W>(c2, launches[big], slabs, s, cap_blocks, hard1, staged_cap, d->staging);
                    for (size_t i = 0; i < launches.size(); ++i)
                        if (static_cast<int>(i) != big) launch_check_class<MsgT, W>(c2, launches[i], slabs, d->side, cap_blocks, hard1, staged_cap, d->staging);
                    MLD_CUDA(cudaEventRecord(d->ev_join, d->side));
                    MLD_CUDA(cudaStreamWaitEvent(s, d->ev_join, 0));
                }
                MLD_LAUNCHED("k_check_update");
                if (h.n_core > 0) {
                    VnArgs v2 = va;
                    v2.want_bits = 1;
                    k_var_update<MsgT, W><<<vn_grid, kBlock, 0, s>>>(v2);
                    MLD_LAUNCHED("k_var_update");
                }
            }
            uint32_t *fcur = d->fail + static_cast<size_t>(parity) * slabs * DW;
            uint32_t *fnext = d->fail + static_cast<size_t>(1 - parity) * slabs * DW;
            if (h.n_cn > 0) {
                SynArgs s2 = sa;
                s2.et = 1;
                s2.hb1 = d->hb1 + static_cast<size_t>(parity) * h1;
                s2.fail = fcur;
                k_syndrome_check<W><<<syn_grid, kBlock, 0, s>>>(s2);
                MLD_LAUNCHED("k_syndrome_check");
            }
            const int32_t nw = slabs * DW;
            k_lane_update_dev<W><<<(std::max(batch, nw) + 127) / 128, 128, 0, s>>>(d->done, fcur, fnext, nw, d->iters,
                                                                                 d->conv, batch, d->lctr, off);
            MLD_LAUNCHED("k_lane_update");
            return MLD_OK;
        };
        // the loop graph of this batch size, variant and layering (built once)
        const int variant = (d->schedule == MLD_SCHED_LAYERED ? 2 : 0) + (hard1 ? 1 : 0);
        cudaGraphExec_t exec = nullptr;
        for (const auto &lg : d->loops)
            if (lg.batch == batch && lg.variant == variant && lg.layers_gen == g->layers_gen) exec = lg.exec;
        if (!exec) {
            cudaGraph_t gr = nullptr;
            MLD_CUDA(cudaGraphCreate(&gr, 0));
            cudaGraphConditionalHandle hnd;
            cudaError_t e = cudaGraphConditionalHandleCreate(&hnd, gr, 1, cudaGraphCondAssignDefault);
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = hnd;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            if (e == cudaSuccess) e = cudaGraphAddNode(&node, gr, nullptr, nullptr, 0, &np);
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(d->cap, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaGraphDestroy(gr);
                return cuda_fail(e, "device loop: graph set-up");
            }
            int s = enqueue_half(1, 1, d->cap);
            if (s == MLD_OK) s = enqueue_half(0, 2, d->cap);
            if (s == MLD_OK) {
                k_loop_cond<W><<<1, 32, 0, d->cap>>>(d->done, slabs * DW, d->lctr, hnd);
                e = cudaGetLastError();
                if (e != cudaSuccess) s = cuda_fail(e, "k_loop_cond");
            }
            cudaGraph_t body = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(d->cap, &body);
            if (s == MLD_OK && ec != cudaSuccess) s = cuda_fail(ec, "device loop: capture");
            if (s == MLD_OK) {
                e = cudaGraphInstantiate(&exec, gr, 0);
                if (e != cudaSuccess) s = cuda_fail(e, "device loop: instantiate");
            }
            cudaGraphDestroy(gr);
            if (s != MLD_OK) return s;
            if (d->loops.size() >= 8) {  // keep the last few batch sizes
                cudaGraphExecDestroy(d->loops.front().exec);
                d->loops.erase(d->loops.begin());
            }
            d->loops.push_back({batch, variant, g->layers_gen, exec});
        }
        {
            int s = timed_launch(d, kClsLayout, st, "k_loop_init", [&] {
                k_loop_init<W><<<(slabs * DW + 127) / 128, 128, 0, st>>>(d->done, slabs, batch, d->lctr, iters);
            });
            if (s != MLD_OK) return s;
        }
        MLD_CUDA(cudaMemsetAsync(d->fail, 0, sizeof(uint32_t) * 2 * slabs * DW, st));
        d->sample_now = true;
        {
            // the whole loop is timed as one region of the check class
            int s = timed_launch(d, kClsCheck, st, "device loop", [&] { cudaGraphLaunch(exec, st); });
            if (s != MLD_OK) return s;
        }
        iters = 0;  // the host loops below do nothing
    }

    if (d->schedule == MLD_SCHED_LAYERED) {
        // layered schedule: layer after layer, each launch updates messages
        // and posteriors in place; decisions after the last iteration (every
        // iteration under early termination)
        const int64_t n_launch = static_cast<int64_t>(g->layer_launches.size());
        for (int32_t l = 1; l <= iters; ++l) {
            const bool last = (l == iters);
            ca.final_pass = (last || et) ? 1 : 0;
            ca.hb1 = hb1_of(l);
            d->sample_now = ((l - 1) % d->timing_every) == 0;
            int s = timed_launch(d, kClsCheck, st, "k_check_layered", [&] {
                CnArgs la = ca;
                la.col = g->lcol;  // layered edge numbering
                for (const mld::LayerLaunch &ll : g->layer_launches) {
                    const mld::CheckClass &k = h.classes[ll.cls];
                    la.cptr = g->leptr + ll.p0;
                    // one wave: the kernels loop over the launch's checks
                    const int blocks = std::max(1, std::min(grid_x(static_cast<int64_t>(ll.count) * TPC),
                                                            sm_count * kLayeredBlocksPerSm));
                    ClassLaunch cl{k.c0, ll.count, k.dc, k.dc + k.dd, ll.e0, k.s0, blocks};
                    launch_layered<MsgT, W>(la, cl, g->lchk + ll.p0, slabs, st, hard1);
                }
            }, static_cast<int>(n_launch));
            if (s != MLD_OK) return s;
            if (last || et) {
                if (h.n_core > 0) {
                    s = timed_launch(d, kClsVar, st, "k_hard_bits", [&] {
                        k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(h.n_core) * (W / 8)), slabs), kBlock, 0,
                                         st>>>(d->Lv, h.n_core, d->hb_core);
                    });
                    if (s != MLD_OK) return s;
                }
                s = syndrome_round(l, et);
                if (s != MLD_OK) return s;
            }
        }
        iters = 0;  // the flooding loop below does nothing
    }
    for (int32_t l = 1; l <= iters; ++l) {
        const bool last = (l == iters);
        ca.final_pass = (last || et) ? 1 : 0;
        ca.hb1 = hb1_of(l);
        ca.hb1_prev = hb1_of(l - 1);
        ca.fail_prev = d->fail + static_cast<size_t>((l - 1) & 1) * slabs * DW;
        ca.fuse = (fused && l >= 2) ? 1 : 0;
        d->sample_now = ((l - 1) % d->timing_every) == 0;
        if (ca.fuse) MLD_CUDA(cudaMemsetAsync(ca.fail_prev, 0, sizeof(uint32_t) * slabs * DW, st));
        if (acc_mode && h.n_core > 0) {
            ca.Lv = acc_of(l - 1);
            ca.acc = acc_of(l);
            int s = timed_launch(d, kClsVar, st, "k_copy4", [&] {
                k_copy4<<<copy_blocks, kBlock, 0, st>>>(reinterpret_cast<float4 *>(ca.acc),
                                                       reinterpret_cast<const float4 *>(d->lch), acc_n4);
            });
            if (s != MLD_OK) return s;
        }
        {
            int s = timed_launch(d, kClsCheck, st, "k_check_update", [&] {
                if (big < 0) {
                    for (const ClassLaunch &cl : launches) launch_check_class<MsgT, W>(ca, cl, slabs, st, cap_blocks, hard1, staged_cap, d->staging);
                    return;
                }
                // the largest class on the caller's stream; the others on the
                // side stream, whose blocks fill the SMs as its last wave
                // drains (errors of the event calls surface as the launch error)
                cudaEventRecord(d->ev_fork, st);
                cudaStreamWaitEvent(d->side, d->ev_fork, 0);
                launch_check_class<MsgT, W>(ca, launches[big], slabs, st, cap_blocks, hard1, staged_cap, d->staging);
                for (size_t i = 0; i < launches.size(); ++i)
                    if (static_cast<int>(i) != big) launch_check_class<MsgT, W>(ca, launches[i], slabs, d->side, cap_blocks, hard1, staged_cap, d->staging);
                cudaEventRecord(d->ev_join, d->side);
                cudaStreamWaitEvent(st, d->ev_join, 0);
            }, static_cast<int>(launches.size()));
            if (s != MLD_OK) return s;
        }
        if (ca.fuse) {  // codewords whose iteration l-1 satisfied every check stop there
            int s = timed_launch(d, kClsSyn, st, "k_lane_update", [&] {
                k_lane_update<W><<<lane_blocks, 128, 0, st>>>(d->done, ca.fail_prev, d->iters, d->conv, batch,
                                                               l - 1, 1);
            });
            if (s != MLD_OK) return s;
        }
        va.want_bits = (last || (et && !fused)) ? 1 : 0;
        if (acc_mode) {
            // the check pass has formed L_v; the last iteration's decisions
            if (last && h.n_core > 0) {
                int s = timed_launch(d, kClsVar, st, "k_hard_bits", [&] {
                    k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(h.n_core) * (W / 8)), slabs), kBlock, 0, st>>>(
                        d->Lv, h.n_core, d->hb_core);
                });
                if (s != MLD_OK) return s;
            }
        } else if (h.n_core > 0) {
            int s = timed_launch(d, kClsVar, st, "k_var_update", [&] {
                k_var_update<MsgT, W><<<vn_grid, kBlock, 0, st>>>(va);
            });
            if (s != MLD_OK) return s;
        }
        if ((et && !fused) || last) {
            int s = syndrome_round(l, et);
            if (s != MLD_OK) return s;
        }
    }

    d->sample_now = true;
    OutArgs oa{g->unit, h.n_vn, h.n_core, h.n_deg1, batch, d->Lv, d->post1, d->hb1, d->iters, h1, bits, post,
               d->scale_out};
    if (h.n_vn > 0) {
        int s = timed_launch(d, kClsLayout, st, "k_deinterleave_out", [&] {
            k_deinterleave_out<W><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(oa);
        });
        if (s != MLD_OK) return s;
    }
    const cudaMemcpyKind kind = out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    MLD_CUDA(cudaMemcpyAsync(conv_out, d->conv, batch, kind, st));
    MLD_CUDA(cudaMemcpyAsync(iters_out, d->iters, sizeof(int32_t) * batch, kind, st));
    return MLD_OK;
}

template <typename MsgT>
int dispatch_w(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syn, int32_t batch,
               int32_t iters, bool et, uint8_t *bits, float *post, uint8_t *conv, int32_t *it,
               cudaStream_t st, bool out_dev) {
    switch (d->W) {
        case 8: return run_decode<MsgT, 8>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        case 16: return run_decode<MsgT, 16>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        case 32: return run_decode<MsgT, 32>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        case 64: return run_decode<MsgT, 64>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        default: return mld::fail(MLD_EINVAL, "unsupported slab width");
    }
}

}  // namespace
