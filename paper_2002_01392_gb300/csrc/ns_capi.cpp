// Navier-Stokes entry points (filled in by the NS kernels).
#include "internal.hpp"

using namespace fcns;

#define FC_NOT_YET(name)                              \
  {                                                   \
    set_error(name ": not available in this build");  \
    return FC_ERR_UNSUPPORTED;                        \
  }

extern "C" {
fc_status ns_params_default(ns_params* p) FC_NOT_YET("ns_params_default")
fc_status ns_workspace_bytes(const ns_params*, size_t*) FC_NOT_YET("ns_workspace_bytes")
fc_status ns_create(const ns_params*, void*, size_t, ns_sim_t*) FC_NOT_YET("ns_create")
fc_status ns_destroy(ns_sim_t) FC_NOT_YET("ns_destroy")
fc_status ns_set_fields(ns_sim_t, const void*, fc_stream_t) FC_NOT_YET("ns_set_fields")
fc_status ns_get_fields(ns_sim_t, void*, fc_stream_t) FC_NOT_YET("ns_get_fields")
fc_status ns_get_state(ns_sim_t, void*, fc_stream_t) FC_NOT_YET("ns_get_state")
fc_status ns_put_state(ns_sim_t, const void*, fc_stream_t) FC_NOT_YET("ns_put_state")
fc_status ns_get_wall_gradp(ns_sim_t, void*, fc_stream_t) FC_NOT_YET("ns_get_wall_gradp")
fc_status ns_put_wall_gradp(ns_sim_t, const void*, fc_stream_t) FC_NOT_YET("ns_put_wall_gradp")
fc_status ns_rhs(ns_sim_t, const void*, void*, fc_stream_t) FC_NOT_YET("ns_rhs")
fc_status fc_poisson_project(ns_sim_t, double, const void*, void*, void*, fc_stream_t) FC_NOT_YET("fc_poisson_project")
fc_status rk_step(ns_sim_t, double, fc_stream_t) FC_NOT_YET("rk_step")
fc_status ns_diagnostics(ns_sim_t, double*, double*, double*, double*, double*, fc_stream_t) FC_NOT_YET("ns_diagnostics")
}
