/* ag.h — C ABI of the GB300 multirotor fleet simulator (libaerialgb).
 *
 * One context simulates n_envs independent environments, each holding one
 * multirotor (quad, hexa or octo) and up to AG_MAX_OBSTACLES static oriented
 * boxes. The operations follow the problem statement of Kulkarni, Forgaard,
 * Alexis, "Aerial Gym - Isaac Gym Simulator for Aerial Robots" (arXiv
 * 2305.16510):
 *   - Sec. III: a gym-style step / reset interface with access to each robot's
 *     position, orientation, linear and angular velocity, and to the obstacle
 *     state;
 *   - Sec. IV-A (Eqs. 1-5) and IV-B (Eqs. 6-9): attitude and velocity command
 *     interfaces of the parallel SE(3) geometric controller; Sec. I: position
 *     tracking in the inertial frame;
 *   - Sec. V: environments are reset with a fresh random draw.
 *
 * Conventions that hold for every entry point:
 *   - World frame z up, g = (0, 0, -9.81) m/s^2. Quaternions are (w, x, y, z),
 *     Hamilton, body -> world. Angular velocity is in the body frame.
 *   - Arrays are structure-of-arrays over environments: field r of env i sits
 *     at index r * n_envs + i, in float32 unless stated.
 *   - Pointer arguments may point to host memory (pageable or pinned) or to
 *     device memory of the context's device; the library copies with
 *     cudaMemcpyAsync(cudaMemcpyDefault). The caller owns them; they are only
 *     borrowed for the duration of the call, except that copies FROM a
 *     pageable host buffer have completed when the call returns, and copies
 *     INTO any buffer have completed once the context's stream has been
 *     synchronised (ag_synchronize) — pinned/device destinations may still be
 *     written after the call returns.
 *   - Calls are asynchronous on the context's CUDA stream unless stated.
 *   - Errors: AG_ERR_INVALID leaves the context unchanged. After a CUDA error
 *     the context is failed and every later call except ag_last_error and
 *     ag_destroy returns AG_ERR_STATE. No C++ exception crosses this ABI.
 */
#ifndef AG_H
#define AG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AG_ABI_VERSION 2
#define AG_MAX_OBSTACLES 64
/* Largest fleet of one context or one serving request: every field index
 * r * n_envs + i of the structure-of-arrays buffers (at most 13 rows) fits
 * in 32 bits, which the kernels' index arithmetic uses. */
#define AG_MAX_ENVS (1u << 28)
#define AG_STATE_DIM 13  /* p.xyz, v.xyz, q.wxyz, Omega.xyz */
#define AG_MAX_ROTORS 8

typedef struct ag_ctx ag_ctx; /* opaque, owned by the library */

typedef enum {
  AG_OK = 0,
  AG_ERR_INVALID = 1,     /* bad argument */
  AG_ERR_OOM = 2,         /* device allocation failed or HBM budget exceeded */
  AG_ERR_CUDA = 3,        /* a CUDA call failed; the context is now failed */
  AG_ERR_STATE = 4,       /* the context failed earlier */
  AG_ERR_TIMEOUT = 5,     /* a bounded wait expired */
  AG_ERR_UNSUPPORTED = 6  /* valid request the library does not implement */
} ag_status;

/* Command interface of one environment (Sec. IV). Targets are four floats:
 *   AG_MODE_POSITION   (p_d.x, p_d.y, p_d.z, psi_d)       world frame, yaw [rad]
 *   AG_MODE_BODY_VEL   (v_d.x, v_d.y, v_d.z, psi_dot_d)   v_d in the yaw-aligned
 *                                                        vehicle frame (Eq. 6)
 *   AG_MODE_ATT_THRUST (phi_d, theta_d, psi_dot_d, f)     Eqs. 1-2, f in newtons
 *   AG_MODE_WRENCH     (f, M_x, M_y, M_z)                 body wrench, bypasses the
 *                                                        controller (still allocated,
 *                                                        clamped and lagged) */
typedef enum {
  AG_MODE_POSITION = 0,
  AG_MODE_BODY_VEL = 1,
  AG_MODE_ATT_THRUST = 2,
  AG_MODE_WRENCH = 3
} ag_mode;

typedef enum { AG_INTEG_SIE = 0 /* semi-implicit Euler */, AG_INTEG_RK4 = 1 } ag_integrator;

typedef struct {
  uint32_t n_envs;            /* 1 .. AG_MAX_ENVS */
  uint32_t substeps_per_step; /* controller + integrator updates per step (1 .. 65536) */
  uint32_t integrator;        /* ag_integrator */
  uint32_t n_obstacles;       /* boxes per environment, 0..AG_MAX_OBSTACLES */
  uint32_t n_quad, n_hexa, n_octo; /* contiguous type ranges in this order; sum == n_envs */
  uint32_t record_every;      /* checkpoint interval K of ag_rollout_loss (0 = 32 steps; <= 65536) */
  float dt;          /* step length [s]; a substep is dt / substeps_per_step */
  float motor_tau;   /* first-order motor time constant [s]; 0 = no lag */
  float drag;        /* linear drag coefficient [N s / m], world frame */
  float sphere_r;    /* collision radius of a vehicle [m] */
  float u_max;       /* per-motor thrust limit [N] (lower limit 0) */
  float arm;         /* rotor distance from the centre [m] */
  float k_yaw;       /* rotor reaction torque per newton of thrust [m] */
  float mass;        /* nominal mass [kg] written at create */
  float inertia[3];  /* nominal diagonal inertia [kg m^2] written at create */
  float kx[3], kv[3], kR[3], kW[3]; /* diagonal controller gains */
  uint64_t seed;     /* Philox key for resets until ag_reset supplies another */
  uint64_t hbm_budget_bytes; /* 0 = no limit; otherwise ag_create fails with
                                AG_ERR_OOM if its buffers would exceed it, and
                                ag_rollout_loss keeps its whole-horizon tape
                                within it (else it uses a one-segment tape) */
} ag_config;

/* Fills *cfg with the defaults of a 1,024-quad fleet: dt 0.01, 1 substep,
 * semi-implicit Euler, no obstacles, tau 0.03, no drag, r 0.2, u_max 5,
 * arm 0.13, k_yaw 0.016, m 0.75, J diag(0.007, 0.007, 0.012),
 * k_x (2,2,3), k_v (2,2,2), k_R (1.2,1.2,0.6), k_Omega (0.2,0.2,0.1), seed 1. */
void ag_config_default(ag_config* cfg);

/* Creates a context on the current CUDA device. `cuda_stream` is a
 * cudaStream_t (NULL = the legacy default stream) that every later call is
 * ordered on. Every environment starts at the origin, level, at rest, motors
 * off, epoch 0, mode AG_MODE_WRENCH with zero targets; call ag_reset to draw
 * initial states. Returns AG_ERR_INVALID for an inconsistent config and
 * AG_ERR_OOM when the buffers do not fit. *out is NULL on failure. */
ag_status ag_create(const ag_config* cfg, void* cuda_stream, ag_ctx** out);

/* Frees every buffer of the context (synchronises its stream first). NULL is
 * accepted. Always AG_OK, also for a failed context. */
ag_status ag_destroy(ag_ctx* ctx);

/* Copies the command of every environment: modes uint8[n_envs] (ag_mode
 * values; any value above 3 acts as AG_MODE_WRENCH) and targets
 * float[4][n_envs] as described at ag_mode. Either pointer may be NULL to
 * keep the current one. Values are not checked (a NaN target propagates into
 * that environment's state only). AG_ERR_CUDA if a copy fails. */
ag_status ag_set_commands(ag_ctx* ctx, const uint8_t* modes, const float* targets);

/* Copies the static obstacles: float[n_obstacles][10][n_envs], per box the
 * centre (3), half-extents (3, > 0) and a UNIT quaternion (4) of its
 * orientation (Sec. V: the obstacle state is privileged information).
 * AG_ERR_INVALID (context unchanged) for a non-finite centre, a half-extent
 * <= 0 or a quaternion whose squared norm is more than 1e-4 from 1; a device
 * array is checked by a kernel, and the call synchronises once. */
ag_status ag_set_obstacles(ag_ctx* ctx, const float* boxes);

/* Copies out the current obstacles float[n_obstacles][10][n_envs] (layout of
 * ag_set_obstacles); they change only when obstacle re-placement is on.
 * AG_ERR_INVALID for a NULL boxes pointer; nothing is copied when the
 * context has no obstacles. */
ag_status ag_get_obstacles(ag_ctx* ctx, float* boxes);

/* Re-placement of one obstacle when its environment resets (Sec. V: the
 * asset manager samples a new position and orientation for every obstacle of
 * a resetting environment; position bounds are fractions of the environment
 * bounds, orientation bounds are Euler angles, and chosen dimensions can be
 * held at a constant value). */
typedef struct {
  float pos_min[3], pos_max[3];     /* fractions in [0, 1] of env_min..env_max, per axis */
  float euler_min[3], euler_max[3]; /* roll, pitch, yaw bounds [rad], within [-pi, pi] */
  uint32_t lock;                    /* bit d set: dimension d (x, y, z, roll, pitch, yaw) is held at fixed[d] */
  float fixed[6];                   /* held values: centre [m] for d < 3, angle [rad] for d >= 3 */
} ag_box_randomization;

/* Enables (per_box non-NULL, n_obstacles host entries) or disables (NULL)
 * the re-placement of obstacles on reset. While enabled, every reset of an
 * environment (ag_reset and collision resets alike) gives each of its boxes k
 * a new centre x_d = env_min_d + (env_max_d - env_min_d) * U[pos_min_d,
 * pos_max_d) and orientation q_z(yaw) q_y(pitch) q_x(roll) with each angle
 * ~ U[euler_min, euler_max), locked dimensions held at fixed[d]; the
 * half-extents are kept. The draws are Philox4x32-10 keyed by the reset seed
 * with counters (env, epoch, k, 1) and (env, epoch, k, 2), transformed in
 * strict binary32, so they are reproducible bit for bit. Host pointers;
 * AG_ERR_INVALID for bounds outside [0, 1] or angles outside [-pi, pi];
 * AG_ERR_OOM (context still usable) if the specification does not fit. */
ag_status ag_set_obstacle_randomization(ag_ctx* ctx, const float env_min[3], const float env_max[3],
                                        const ag_box_randomization* per_box);

/* Depth images of n_cams vehicle-mounted pinhole cameras, rendered by ray
 * casting against each environment's boxes (the paper's depth cameras,
 * Sec. III, and its kernel-based ray casting, Sec. VII). Camera j belongs to
 * environment env_ids[j] (host or device array; NULL = environments 0 ..
 * n_cams-1), sits at p + R cam_offset (host float[3] in the body frame, NULL
 * = the centre of mass) and looks along body +x with body +z up. Pixel
 * (row r, column c) of a width x height image with horizontal field of view
 * hfov [rad] sees along R (1, -(c + 0.5 - width/2) / f, -(r + 0.5 - height/2)
 * / f) with f = (width/2) / tan(hfov/2); its value is the distance along the
 * optical axis to the nearest box surface in front of the camera (0 inside a
 * box), or max_range if none is closer. depth: float[n_cams][height][width],
 * host or device. AG_ERR_INVALID for an empty image, hfov outside (0, pi),
 * max_range <= 0 or an environment id out of range in a host array; an id
 * out of range in a device array is not read through: that camera's image
 * is all NaN. AG_ERR_OOM (context still usable) if the staging buffer of a
 * host destination does not fit. */
ag_status ag_render_depth(ag_ctx* ctx, uint32_t width, uint32_t height, float hfov, float max_range,
                          const float* cam_offset, const uint32_t* env_ids, uint32_t n_cams, float* depth);

/* Copies per-environment rigid-body parameters float[4][n_envs]: mass and
 * the diagonal inertia J_xx, J_yy, J_zz. AG_ERR_INVALID (context unchanged)
 * unless all are finite and > 0; a device array is checked by a kernel, and
 * the call synchronises once. */
ag_status ag_set_body(ag_ctx* ctx, const float* body);

/* Advances every environment by n_substeps substeps (a positive multiple of
 * substeps_per_step) in ONE fused kernel launch: per substep the controller
 * of the environment's mode (Sec. IV), rotor allocation with per-motor clamp
 * to [0, u_max] and first-order motor lag, and one integrator update with
 * quaternion renormalisation; after the last substep of every step the
 * vehicle sphere is tested against every box of its environment, and an
 * environment that touches one is reset in place (epoch + 1, Philox draw of
 * a new state, as ag_reset). A vehicle's test is skipped while it has moved
 * less from its last exact test than that test's clearance to the nearest
 * box, minus a slack far above float32 rounding: such a test could not hit,
 * so every decision is the one the exact test makes at every step. Afterwards the collided flags mark environments
 * that hit a box in any step of this call and the reset list holds each
 * environment reset during this call once (order unspecified).
 * AG_ERR_INVALID unless n_substeps / substeps_per_step is in 1 .. 2^31 - 1.
 * The call allocates nothing and never synchronises, so a loop of calls can
 * be captured in a CUDA graph on the context's stream (make one call outside
 * the capture first: it sets the kernel's shared-memory attribute). */
ag_status ag_step(ag_ctx* ctx, uint32_t n_substeps);

/* Same results as ag_step, computed by one kernel launch per stage per
 * substep (controller, allocation, integrator) and per step (collision,
 * reset), with every intermediate written to and read back from device
 * memory. It is the unfused comparison point; results agree with ag_step to
 * float32 rounding. Errors as ag_step. */
ag_status ag_step_plain(ag_ctx* ctx, uint32_t n_substeps);

/* The controller stage alone (Sec. IV): for every environment, its command
 * mode and targets, body parameters and the context's gains, writes the
 * commanded collective thrust and moments float[4][n_envs] (f, M_x, M_y,
 * M_z) at the states float[13][n_envs] (NULL = the current states; q need
 * not be unit). Host or device pointers; nothing else changes. For
 * inspecting what the controller asks for, and for testing it on its own.
 * AG_ERR_INVALID for a NULL wrench; AG_ERR_OOM if the staging buffer for a
 * given state does not fit. */
ag_status ag_eval_controller(ag_ctx* ctx, const float* state, float* wrench);

/* Resets the environments whose mask byte is non-zero (mask NULL = all):
 * epoch + 1, then position U[-2, 2)^3 m, attitude a rotation by U[0, pi/6)
 * about a uniformly random axis, velocity N(0, 0.5^2) m/s per axis, zero body
 * rate and every motor at hover thrust m g / n_rot. The draw is Philox4x32-10
 * with key = seed and counter (env, epoch, slot, 0), transformed in strict
 * binary32 arithmetic, so it is reproducible bit for bit. `seed` also becomes
 * the key of later collision resets. Writes the reset list and clears the
 * collided flags. The mask (host or device) is copied; AG_ERR_CUDA if the
 * copy or the launch fails. */
ag_status ag_reset(ag_ctx* ctx, const uint8_t* mask, uint64_t seed);

/* Copies out the state float[13][n_envs] (p, v, q, Omega), the collided
 * flags uint8[n_envs] and the reset list uint32[n_envs] (its first
 * *n_reset entries are valid) of the last ag_step / ag_reset. Any pointer may
 * be NULL. A non-NULL n_reset synchronises the stream. AG_ERR_CUDA if a copy
 * fails. */
ag_status ag_get_state(ag_ctx* ctx, float* state, uint8_t* collided, uint32_t* reset_ids, uint32_t* n_reset);

/* Copies out the motor thrusts float[8][n_envs] (rows >= n_rot unused) and
 * the reset epochs uint32[n_envs]. Either pointer may be NULL. AG_ERR_CUDA if
 * a copy fails. */
ag_status ag_get_motors(ag_ctx* ctx, float* motors, uint32_t* epoch);

/* Overwrites the state float[13][n_envs]; motors float[8][n_envs] and
 * epoch uint32[n_envs] may be NULL to keep the current values. With
 * ag_get_state / ag_get_motors this checkpoints and resumes a fleet bit for
 * bit. Values are not checked. AG_ERR_INVALID for a NULL state. */
ag_status ag_set_state(ag_ctx* ctx, const float* state, const float* motors, const uint32_t* epoch);

/* Allocation-free unfused step: the computation of ag_step_plain, without a
 * context and without allocating any device memory.
 *
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc: for example a simulator embedded in a real-time
 * control loop, where cudaMalloc's implicit device synchronisation and
 * unbounded latency are forbidden once the loop runs, or a host application
 * that owns the whole device-memory budget and does not let libraries
 * allocate. The caller passes every input and output as device pointers in
 * the layouts of ag_get_state / ag_get_motors / ag_set_commands /
 * ag_set_obstacles / ag_set_body; state, motors and epoch are updated in
 * place, collided / reset_ids / *n_reset (n_reset is a device pointer)
 * describe this call, and `seed` keys the collision resets. The intermediate
 * wrenches, hit bytes and reset counters live in a static device array sized
 * for AG_NOALLOC_MAX_ENVS environments (2,424,832 bytes), which every GPU that
 * loads the library holds until the process exits.
 *   - Two differences from a context's ag_step_plain: a collision reset never
 *     re-draws the environment's obstacles (there is no
 *     ag_set_obstacle_randomization here), and the body array is not checked
 *     (ag_set_body rejects non-finite or non-positive masses and inertias;
 *     here they are the caller's precondition).
 *   - n_envs > AG_NOALLOC_MAX_ENVS, an invalid config, an n_substeps that is
 *     not a positive multiple of substeps_per_step, a NULL pointer, a pointer
 *     to host memory or to another device's memory, or a stream of another
 *     device returns AG_ERR_INVALID ("another device" means other than the
 *     current one, cudaGetDevice). A CUDA failure returns AG_ERR_CUDA. The
 *     reason is written to err (err_len bytes, may be NULL).
 *   - The array's address belongs to the CUDA context current at the call
 *     (the primary context, or a context the host application made current).
 *     Every call outside stream capture looks the address up in that context
 *     (cudaGetSymbolAddress; the first lookup in a context loads the module)
 *     and remembers it for that context. A call on a stream that is being
 *     captured uses the remembered address, so make one call in each context
 *     (and again after cudaDeviceReset) before any capture begins; without
 *     one the call returns AG_ERR_STATE.
 *   - Every call in a context shares the one array and leaves its contents
 *     behind; the call clears what must start at zero itself. Two calls whose
 *     work overlaps on the GPU (for example on two streams) race on the array
 *     and give undefined results: order them on one stream. */
#define AG_NOALLOC_MAX_ENVS 65536
ag_status ag_step_plain_noalloc(const ag_config* cfg, void* cuda_stream, uint32_t n_substeps, uint64_t seed,
                                float* state, float* motors, const float* body, const uint8_t* modes,
                                const float* targets, const float* boxes, uint32_t* epoch, uint8_t* collided,
                                uint32_t* reset_ids, uint32_t* n_reset, char* err, size_t err_len);

/* Sets the 12 diagonal controller gains (k_x, k_v, k_R, k_Omega, three each,
 * in that order) used by every later launch. gains12 may be a host or device
 * pointer (the call synchronises the copy). AG_ERR_INVALID (gains unchanged)
 * for NULL or a non-finite gain. */
ag_status ag_set_gains(ag_ctx* ctx, const float* gains12);

/* Differentiable rollout, forward half. Advances every environment n_steps
 * steps from its current state with the controller of its command mode
 * (position tracking, Sec. I after Lee et al. 2011; body velocity, Eqs. 6-9;
 * attitude and thrust, Eqs. 1-2; each with the attitude law of Sec. IV-A
 * Eqs. 3-5; or a direct wrench), allocation with clamp and lag, and
 * semi-implicit Euler, without collision tests; records a checkpoint (state +
 * motors) every record_every steps; and writes
 *   loss[i] = sum_{t=1..n_steps} w_pos |p_t - p_goal_i|^2 + w_omega |Omega_t|^2
 * (x_t = the state after step t; p_goal float[3][n_envs]). saturated (may be
 * NULL) flags environments in which some motor command was clamped during
 * the rollout; there the gradient uses the clamp's subgradient 0. Requires
 * semi-implicit Euler, one substep per step and no obstacles (else
 * AG_ERR_UNSUPPORTED); AG_ERR_INVALID for n_steps outside 1 .. 2^30, NULL
 * p_goal or loss; AG_ERR_OOM (context still usable) when the checkpoints do
 * not fit. Does not synchronise. Commands, body parameters and gains must not
 * change until ag_backward has run. */
ag_status ag_rollout_loss(ag_ctx* ctx, uint32_t n_steps, float w_pos, float w_omega, const float* p_goal,
                          float* loss, uint8_t* saturated);

/* Differentiable rollout, reverse half: the hand-written adjoint of the last
 * ag_rollout_loss. With weights c_i = loss_weights[i] (NULL = all 1), writes
 * the gradient of sum_i c_i loss[i] with respect to each environment's
 * initial state float[13][n_envs] (grad_x0), with respect to the 12 gains
 * float[12] (grad_gains, the fleet sum, reduced in a fixed order so repeated
 * calls give identical bits), optionally each environment's share
 * float[12][n_envs] (grad_gains_per_env), and with respect to each
 * environment's four command targets float[4][n_envs] (grad_targets, in the
 * target order of ag_mode: angles in radians, yaw rate in rad/s). Any output
 * may be NULL. The gradient with respect to the initial quaternion is that of
 * the loss as a function of q_0 / |q_0|. Where the controller meets a
 * degenerate direction (zero commanded acceleration, thrust along the
 * heading, body x axis vertical) the gradient is that of the fallback
 * branch. Returns AG_ERR_STATE if nothing was recorded.
 * The reverse sweep needs every step's start state again. ag_rollout_loss
 * allocates a tape of the whole horizon (n_steps x 21 floats per
 * environment) when it fits in device memory and in hbm_budget_bytes; then
 * one launch recomputes every checkpoint segment's states into it in
 * parallel before the sweep. Otherwise the tape holds one segment
 * (record_every x 21 floats per environment) and the sweep recomputes the
 * segments one after another. The two agree to float32 rounding. */
ag_status ag_backward(ag_ctx* ctx, const float* loss_weights, float* grad_x0, float* grad_gains,
                      float* grad_gains_per_env, float* grad_targets);

/* ------------------------------------------------------------------------
 * Reach-a-setpoint task (Sec. I: policies learn to fly the vehicle to a goal
 * setpoint through the attitude or velocity command interface).
 *
 * One task step maps the policy's actions to every environment's command,
 * advances the fleet one step (ag_step with substeps_per_step substeps,
 * collision resets included) and then, per environment i with goal g_i:
 *   reward  = -crash                                  if it collided
 *             -|p - g| - w_v |v| - w_omega |Omega|    otherwise
 *   done    = collided or |p - g| > max_dist or steps >= max_steps
 *             (steps counts the episode's steps, this one included)
 * An episode that ended without a collision is reset in place exactly as
 * ag_reset draws it (a collision already reset it inside the step), and the
 * step counter of every ended episode returns to 0. The observation then
 * describes the state the policy acts on next (after any reset):
 *   obs[i] = (p - g (3), v (3), q (w, x, y, z) with w >= 0 (4), Omega (3))
 * One kernel launch does all of it per environment; nothing synchronises
 * and nothing is allocated after ag_reach_begin, so a training loop can
 * capture ag_reach_step in a CUDA graph on the context's stream (a stream
 * other than the legacy default one) and replay it; replays give the same
 * bits as direct calls.
 * ------------------------------------------------------------------------ */
typedef struct ag_reach_config {
  uint32_t command_mode;   /* AG_MODE_ATT_THRUST or AG_MODE_BODY_VEL */
  float action_scale[4];   /* command_k = action_offset[k] + action_scale[k] * clamp(a_k, -1, 1) */
  float action_offset[4];  /* (targets as at ag_mode: attitude (phi, theta, psi_dot, f), velocity (v, psi_dot)) */
  float w_v;               /* reward weight of the speed |v| [1/(m/s)] */
  float w_omega;           /* reward weight of the body rate |Omega| [1/(rad/s)] */
  float crash;             /* penalty of a collision */
  float max_dist;          /* an episode ends beyond this distance to the goal [m] */
  uint32_t max_steps;      /* an episode ends after this many steps (>= 1) */
} ag_reach_config;

/* Attitude interface for the default 0.75 kg quad: roll and pitch within
 * +-pi/6, yaw rate within +-1 rad/s, thrust m g (1 +- 0.5); w_v 0.1,
 * w_omega 0.01, crash 10, max_dist 8 m, max_steps 500. */
void ag_reach_config_default(ag_reach_config* cfg);

/* Starts the task: every environment's mode becomes cfg->command_mode, the
 * goals float[3][n_envs] (host or device) are copied and every step counter
 * is set to 0. States are left as they are (call ag_reset first for fresh
 * episodes). AG_ERR_INVALID for another mode, max_steps 0, a negative weight
 * or penalty, max_dist <= 0 or goals NULL; AG_ERR_OOM (context still usable)
 * if the goals and step counters do not fit. */
ag_status ag_reach_begin(ag_ctx* ctx, const ag_reach_config* cfg, const float* goals);

/* One task step. actions: device float[n_envs][4], 16-byte aligned. obs:
 * device float[n_envs][13]; reward: device float[n_envs]; done: device
 * uint8[n_envs]. The collision resets use the context's reset seed (that of
 * the last ag_reset, else the config's). The collided flags (ag_get_state)
 * describe this step; the reset list is not updated (done marks every
 * episode that ended). AG_ERR_STATE before ag_reach_begin; AG_ERR_INVALID
 * for a NULL or misaligned pointer. */
ag_status ag_reach_step(ag_ctx* ctx, const float* actions, float* obs, float* reward, uint8_t* done);

/* Observations float[n_envs][13] (device) of the current states, as written
 * by ag_reach_step; nothing else changes. AG_ERR_STATE before ag_reach_begin. */
ag_status ag_reach_observe(ag_ctx* ctx, float* obs);

/* ------------------------------------------------------------------------
 * Continuous-batching rollout server.
 *
 * A server owns one device slab of hbm_budget_bytes (allocated once at
 * creation) and a persistent host thread. Each submitted request is a whole
 * rollout of an independent quadrotor fleet (its own size, horizon, command
 * mode per environment, obstacle count and Philox seed). The thread admits
 * requests first-in first-out while a slot (max_active) and slab memory are
 * free, draws their initial states (as ag_reset), and advances ALL active
 * requests together: one kernel launch covers every environment of every
 * active request for chunk_steps steps (fewer for a request's last chunk),
 * with the same per-step computation as ag_step (controller, allocation,
 * integrator, collision test, Philox reset). Requests that arrive while
 * others run join at the next launch; their state stays on the device until
 * they finish. A finished request's final state and reset epochs are kept
 * on the host until ag_server_wait collects them. Chunk boundaries are
 * counted from each request's own first launch, so a request's result is
 * bit-identical alone or in any mix, and to ag_step calls of chunk_steps
 * steps each on the same inputs (every fused multiply-add of the step is
 * explicit in the source, so both kernels round alike). max_active = 1
 * makes the same loop run one request per launch (the unbatched comparison
 * point). Physics settings
 * (integrator, substeps, dt, gains, motor model, radius) come from `physics`;
 * its fleet-size fields are ignored. */
#define AG_SERVER_MAX_ACTIVE 4096

typedef struct ag_server ag_server;

typedef struct {
  ag_config physics;         /* per-step physics of every request */
  uint32_t max_active;       /* requests on the device at once, 1..AG_SERVER_MAX_ACTIVE */
  uint32_t chunk_steps;      /* steps per launch (1 .. 2^30) */
  uint64_t hbm_budget_bytes; /* device memory for request buffers (>= 1 MiB) */
} ag_server_config;

typedef struct {
  uint32_t n_envs;           /* quadrotors in this request (>= 1) */
  uint32_t n_steps;          /* horizon in steps (>= 1) */
  uint32_t n_obstacles;      /* boxes per environment, 0..AG_MAX_OBSTACLES */
  uint32_t reserved;
  uint64_t seed;             /* Philox key of its initial draw and collision resets */
  const uint8_t* modes;      /* [n_envs] ag_mode values */
  const float* targets;      /* [4][pitch]: first n_envs of each row used */
  const float* body;         /* [4][pitch] m, J diagonal; NULL = the physics' nominal body */
  const float* boxes;        /* [n_obstacles * 10][pitch] as ag_set_obstacles; NULL if none */
  uint64_t pitch;            /* row stride of targets/body/boxes in elements (0 = n_envs) */
} ag_request;

typedef struct {
  uint64_t launches;         /* chunk launches so far */
  uint64_t completed;        /* requests finished */
  uint64_t pending;          /* waiting for admission */
  uint64_t active;           /* on the device */
  double vehicle_steps;      /* environment-steps computed */
  double gpu_ms;             /* summed device time of the launches (CUDA events) */
  uint64_t hbm_used_bytes;   /* slab bytes held by active requests */
} ag_server_stats;

/* Defaults: RK4 with 4 substeps of 2.5 ms, the ag_config_default body,
 * motor model and gains, max_active 1024, chunk_steps 50, a 40 GiB budget. */
void ag_server_config_default(ag_server_config* cfg);

/* Creates a server on the current CUDA device and starts its loop thread.
 * AG_ERR_INVALID for a bad config, AG_ERR_OOM if the slab does not fit. */
ag_status ag_server_create(const ag_server_config* cfg, ag_server** out);

/* Queues a request (thread-safe, non-blocking) and returns its id. The input
 * arrays (host or device) must stay valid until ag_server_wait has returned
 * for this id. The loop uploads them when it admits the request: device (or
 * pinned) arrays are copied asynchronously, while pageable host arrays make
 * the loop wait for their copy before it queues the next chunk. Their contents are not checked (submission stays cheap): they
 * must meet the preconditions of ag_set_commands, ag_set_body and
 * ag_set_obstacles. AG_ERR_INVALID for a malformed request (n_envs outside
 * 1 .. AG_MAX_ENVS, other counts, NULL arrays, pitch), AG_ERR_OOM if it
 * could never fit the budget, AG_ERR_STATE
 * if the server has failed. */
ag_status ag_server_submit(ag_server* s, const ag_request* req, uint64_t* id);

/* Blocks until request `id` finishes or timeout_s seconds pass
 * (AG_ERR_TIMEOUT; the request stays queued and can be waited for again).
 * On success copies its final state float[13][n_envs] and reset epochs
 * uint32[n_envs] into HOST buffers (either may be NULL), writes its latency
 * from submission to completion in milliseconds, and forgets the request. */
ag_status ag_server_wait(ag_server* s, uint64_t id, double timeout_s, float* final_state, uint32_t* epoch,
                         double* latency_ms);

/* Snapshot of the server's counters (thread-safe). AG_ERR_INVALID for a NULL
 * server or out. */
ag_status ag_server_get_stats(ag_server* s, ag_server_stats* out);

/* Stops the loop after the requests on the device finish, abandons queued
 * ones, and frees everything. NULL is accepted; always AG_OK. */
ag_status ag_server_destroy(ag_server* s);

/* Waits for all work queued on the context's stream. */
ag_status ag_synchronize(ag_ctx* ctx);

/* Number of environments / the configuration the context was created with
 * (the gains as last set). AG_ERR_INVALID for a NULL ctx or out. */
ag_status ag_get_config(const ag_ctx* ctx, ag_config* out);

/* Fault injection for testing a caller's error handling: marks the context
 * failed exactly as a CUDA error would (message: why, or "injected failure"),
 * without touching the device. Later calls return AG_ERR_STATE as described
 * above. AG_ERR_INVALID for a NULL ctx. */
ag_status ag_inject_failure(ag_ctx* ctx, const char* why);

/* Message of the last error of this context ("" if none); valid until the
 * next call on the context. NULL ctx gives the last ag_create failure. */
const char* ag_last_error(const ag_ctx* ctx);

/* AG_ABI_VERSION of the loaded library. */
int ag_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AG_H */
