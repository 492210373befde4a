/*
 * render_oracle.h -- CPU restatement of the headless rendering of the
 * simulated state (the paper's visualisation options, Sec. 3: colormaps of
 * eta, u, v and the speed, photorealistic water by the Fresnel equations,
 * a terrain colormap and a grid overlay), written into an RGBA image.
 *
 * TEST INFRASTRUCTURE ONLY: the plain reference the CUDA renderer is checked
 * against, byte for byte.  All shading arithmetic is IEEE single precision,
 * one rounded operation at a time (add, subtract, multiply, divide, square
 * root; no fused multiply-add, no transcendental functions), so that any
 * correct implementation of the same sequence gives the same bytes.
 *
 * Inputs are interior, row-major [ny][nx] arrays (w, P, Q and the cell bed
 * Bbar), converted to single precision; the image is [ny][nx][4] bytes, row
 * j of the image being grid row j (south first).
 */
#ifndef RENDER_ORACLE_H
#define RENDER_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { RO_ETA = 0, RO_U = 1, RO_V = 2, RO_SPEED = 3, RO_FRESNEL = 4 };

typedef struct {
    int mode;             /* RO_*                                              */
    float vmin, vmax;     /* colormap range of the shown value (modes 0-3)     */
    float dry_h;          /* a cell is land where w - Bbar <= dry_h            */
    float h_min;          /* velocities u = P / max(h, h_min)                  */
    float zmin, zmax;     /* terrain colormap range of the bed elevation       */
    float grid;           /* grid line spacing [m]; 0 draws none               */
    float exaggeration;   /* vertical scale of the surface and bed normals     */
    float view[3];        /* direction of view, towards the surface (z < 0)    */
    float sun[3];         /* direction towards the light, for the terrain      */
    float absorb;         /* refraction: bed colour weight 1 / (1 + absorb h)  */
} ro_params;

void ro_render(int nx, int ny, double dx, double dy, double ws, const double *w, const double *P,
               const double *Q, const double *Bbar, const ro_params *p, unsigned char *rgba);

/* building blocks, for the pins */
float ro_fresnel(float cos_i);                       /* unpolarised, air -> water */
void ro_colormap(int which, float t, float rgb[3]);  /* 0 diverging, 1 sequential, 2 terrain */

#ifdef __cplusplus
}
#endif
#endif
